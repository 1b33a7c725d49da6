// C ABI of the KFBI library and its host orchestration: handle lifecycle,
// the boundary integral operator A psi (Algorithm 1), GMRES / simple
// iteration on A psi = g (Section 4), the Neumann solve and the Strang step
// (Section 3).  All arithmetic runs in the kernels of dst.cu, ops.cu and
// setup.cu; the host only sequences launches and reads one residual estimate
// per Krylov iteration, one iteration behind the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace kfbi {

static thread_local char g_err[1024] = "";
std::atomic<long long> g_launches{0};

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int small_size(int m);
int small_res(int m);
int small_g(int m);
int small_hcol(int m);
int small_nrm2(int m);
int small_y(int m);
int arnoldi_add(kfbi_handle* h, double* small, int m, int n);
int launch_init_arnoldi(kfbi_handle* h, double* small, int m);

namespace {

// nodes of a field (user layout): (N-1)^d interior nodes of the Dirichlet
// box, all (N+1)^d nodes of the Neumann box
int64_t grid_points(const kfbi_handle* h) { return field_count(h->grid); }

int64_t interior_points(const kfbi_handle* h) {
  const int64_t n1 = h->grid.N - 1;
  return h->grid.dim == 3 ? n1 * n1 * n1 : n1 * n1;
}

// nodes of a work grid: N^d (padded Dirichlet layout) or the (N+1)^d field
// layout of the Neumann box
int64_t padded_points(const kfbi_handle* h) {
  const int64_t P = work_n(h->grid);
  return h->grid.dim == 3 ? P * P * P : P * P;
}

bool neumann_box(const kfbi_handle* h) { return h->grid.bc == KFBI_BOX_NEUMANN; }

// density vector x seen by the correction and jump rows: psi (3-D) or
// [psi; spline moments] (2-D)
int density_vector(kfbi_handle* h, const double* psi, const double** x) {
  if (h->grid.dim == 2) {
    int rc = launch_spline(h, psi, h->w.xvec);
    if (rc) return rc;
    *x = h->w.xvec;
  } else {
    *x = psi;
  }
  return KFBI_OK;
}

// density vector of one component into buf (2-D: [psi; spline moments])
int density_vector_buf(kfbi_handle* h, const double* psi, double* buf, const double** x) {
  if (h->grid.dim == 2) {
    int rc = launch_spline(h, psi, buf);
    if (rc) return rc;
    *x = buf;
  } else {
    *x = psi;
  }
  return KFBI_OK;
}

// Coupled anisotropic system (Eq. pde1 with diagonal conductivities): out =
// base + sgn * A psi for the density pair psi = (psi_i, psi_e) (2M): each
// component's corrections from its own rows (t: D_i, t2: D_e), the coupled
// box solve, each component's conormal limit, and the rank-one term
// (1, 1) <(ds, ds), psi> / (2 |Gamma|) that removes the common-constant null
// space of the coupled Neumann problem.
int apply_A_coupled(kfbi_handle* h, double kappa, const double* psi, double* out, double sgn, const double* base) {
  const int M = h->t.M;
  const double *xi, *xe;
  int rc;
  if ((rc = density_vector_buf(h, psi, h->w.xvec, &xi))) return rc;
  if ((rc = density_vector_buf(h, psi + M, h->w.xvec2, &xe))) return rc;
  if ((rc = launch_correction_t(h, h->t, xi, h->w.corr))) return rc;
  if ((rc = launch_correction_t(h, h->t2, xe, h->w.corr2))) return rc;
  SolveArgs si, se;
  si.corr = h->w.corr;
  se.corr = h->w.corr2;
  Coupling cp = h->cpl;
  cp.kappa = kappa;
  if ((rc = box_solve_coupled64(h, si, se, cp, h->w.grid64, h->w.grid64b))) return rc;
  if ((rc = launch_limit64_t(h, h->t, h->w.grid64, xi, base, sgn, out))) return rc;
  if ((rc = launch_limit64_t(h, h->t2, h->w.grid64b, xe, base ? base + M : nullptr, sgn, out + M))) return rc;
  return launch_rank_one_coupled(h, psi, out, sgn);
}

// g = (gN_i, gN_e) - conormal limits of the coupled box solve of the sources
// (alpha_i src_i, alpha_e src_e); the padded grids keep v_V
int rhs_g_coupled(kfbi_handle* h, double kappa, const double* src_i, double a_i, const double* src_e, double a_e,
                  const double* gNi, const double* gNe, double* g) {
  const int M = h->t.M;
  SolveArgs si, se;
  si.src = src_i;
  si.alpha = a_i;
  se.src = src_e;
  se.alpha = a_e;
  Coupling cp = h->cpl;
  cp.kappa = kappa;
  int rc;
  if ((rc = box_solve_coupled64(h, si, se, cp, h->w.grid64, h->w.grid64b))) return rc;
  if ((rc = launch_limit64_t(h, h->t, h->w.grid64, nullptr, gNi, -1.0, g))) return rc;
  return launch_limit64_t(h, h->t2, h->w.grid64b, nullptr, gNe, -1.0, g + M);
}

// (Phi_i, Phi_e) = v_V + v_B(psi) of the coupled problem in one coupled solve
// of the combined right-hand sides; r (2M, optional) receives the true
// residual g^N - n.D grad u^+ - rank-one term
int assemble_coupled(kfbi_handle* h, double kappa, const double* src_i, double a_i, const double* src_e, double a_e,
                     const double* psi, const double* gNi, const double* gNe, double* phi_i, double* phi_e,
                     double* r) {
  const int M = h->t.M;
  const double *xi, *xe;
  int rc;
  if ((rc = density_vector_buf(h, psi, h->w.xvec, &xi))) return rc;
  if ((rc = density_vector_buf(h, psi + M, h->w.xvec2, &xe))) return rc;
  if ((rc = launch_correction_t(h, h->t, xi, h->w.corr))) return rc;
  if ((rc = launch_correction_t(h, h->t2, xe, h->w.corr2))) return rc;
  SolveArgs si, se;
  si.src = src_i;
  si.alpha = a_i;
  si.corr = h->w.corr;
  si.out_user = phi_i;
  se.src = src_e;
  se.alpha = a_e;
  se.corr = h->w.corr2;
  se.out_user = phi_e;
  Coupling cp = h->cpl;
  cp.kappa = kappa;
  if ((rc = box_solve_coupled64(h, si, se, cp, h->w.grid64, h->w.grid64b))) return rc;
  if (r == nullptr) return KFBI_OK;
  if ((rc = launch_limit64_t(h, h->t, h->w.grid64, xi, gNi, -1.0, r))) return rc;
  if ((rc = launch_limit64_t(h, h->t2, h->w.grid64b, xe, gNe, -1.0, r + M))) return rc;
  return launch_rank_one_coupled(h, psi, r, -1.0);
}

// the coupled A psi with float32 transforms (the inner operator of GMRES-IR;
// the 2 x 2 mode solve and the limits stay float64)
int apply_A_coupled32(kfbi_handle* h, double kappa, const double* psi, double* out, double sgn,
                      const double* base) {
  const int M = h->t.M;
  const double *xi, *xe;
  int rc;
  if ((rc = density_vector_buf(h, psi, h->w.xvec, &xi))) return rc;
  if ((rc = density_vector_buf(h, psi + M, h->w.xvec2, &xe))) return rc;
  if ((rc = launch_correction_t(h, h->t, xi, h->w.corr))) return rc;
  if ((rc = launch_correction_t(h, h->t2, xe, h->w.corr2))) return rc;
  SolveArgs si, se;
  si.corr = h->w.corr;
  se.corr = h->w.corr2;
  Coupling cp = h->cpl;
  cp.kappa = kappa;
  if ((rc = box_solve_coupled32(h, si, se, cp, h->w.grid32, h->w.grid32b))) return rc;
  if ((rc = launch_limit32_t(h, h->t, h->w.grid32, xi, base, sgn, out))) return rc;
  if ((rc = launch_limit32_t(h, h->t2, h->w.grid32b, xe, base ? base + M : nullptr, sgn, out + M))) return rc;
  return launch_rank_one_coupled(h, psi, out, sgn);
}

// float64-accurate coupled box solve from float32 transforms: (u_i, u_e) =
// L_h^{-1}(a_i src_i + corr_i, a_e src_e + corr_e) on the user layout, then
// rounds of the float64 coupled residual, each solved in float32 and added
int refine_rounds(const kfbi_handle* h);
int refined_solve_coupled(kfbi_handle* h, double kappa, const double* src_i, double a_i, const double* src_e,
                          double a_e, const double* corr_i, const double* corr_e, double* ui, double* ue) {
  Coupling cp = h->cpl;
  cp.kappa = kappa;
  SolveArgs si, se;
  si.src = src_i;
  si.alpha = a_i;
  si.corr = corr_i;
  si.out_user = ui;
  se.src = src_e;
  se.alpha = a_e;
  se.corr = corr_e;
  se.out_user = ue;
  // the float grids keep the solution for the first round's float-float
  // residual
  int rc = box_solve_coupled32(h, si, se, cp, h->w.grid32, h->w.grid32b);
  if (rc) return rc;
  const int rounds = refine_rounds(h);
  for (int r = 0; r < rounds; ++r) {
    SolveArgs ri, re;
    if (r == 0) {
      // (u_i, u_e) is exactly the pair of float grids just solved
      if ((rc = launch_residual_ff_coupled(h, src_i, a_i, src_e, a_e, corr_i, corr_e, ui, ue, kappa, h->w.res32,
                                           h->w.res32b)))
        return rc;
      ri.src32 = h->w.res32;
      re.src32 = h->w.res32b;
    } else {
      if ((rc = launch_residual_coupled(h, src_i, a_i, src_e, a_e, corr_i, corr_e, ui, ue, kappa, h->w.res64,
                                        h->w.res64b)))
        return rc;
      ri.src = h->w.res64;
      re.src = h->w.res64b;
    }
    ri.out_user = ui;
    ri.aux = ui;
    ri.gamma = 1.0;
    ri.keep = false;
    re.out_user = ue;
    re.aux = ue;
    re.gamma = 1.0;
    re.keep = false;
    if ((rc = box_solve_coupled32(h, ri, re, cp, h->w.grid32, h->w.grid32b))) return rc;
  }
  return KFBI_OK;
}

// coupled out = base + sgn * A psi with the refined solve (v_B of both
// components left in u64, u64b)
int apply_A_acc_coupled(kfbi_handle* h, double kappa, const double* psi, double* out, double sgn,
                        const double* base) {
  const int M = h->t.M;
  const double *xi, *xe;
  int rc;
  if ((rc = density_vector_buf(h, psi, h->w.xvec, &xi))) return rc;
  if ((rc = density_vector_buf(h, psi + M, h->w.xvec2, &xe))) return rc;
  if ((rc = launch_correction_t(h, h->t, xi, h->w.corr))) return rc;
  if ((rc = launch_correction_t(h, h->t2, xe, h->w.corr2))) return rc;
  if ((rc = refined_solve_coupled(h, kappa, nullptr, 1.0, nullptr, 1.0, h->w.corr, h->w.corr2, h->w.u64, h->w.u64b)))
    return rc;
  if ((rc = launch_limit_user_t(h, h->t, h->w.u64, xi, base, sgn, out))) return rc;
  if ((rc = launch_limit_user_t(h, h->t2, h->w.u64b, xe, base ? base + M : nullptr, sgn, out + M))) return rc;
  return launch_rank_one_coupled(h, psi, out, sgn);
}

// coupled g with the refined volume solve (v_V of both components kept in
// vV64, vV64b)
int rhs_g_acc_coupled(kfbi_handle* h, double kappa, const double* src_i, double a_i, const double* src_e, double a_e,
                      const double* gNi, const double* gNe, double* g) {
  const int M = h->t.M;
  int rc = refined_solve_coupled(h, kappa, src_i, a_i, src_e, a_e, nullptr, nullptr, h->w.vV64, h->w.vV64b);
  if (rc) return rc;
  if ((rc = launch_limit_user_t(h, h->t, h->w.vV64, nullptr, gNi, -1.0, g))) return rc;
  return launch_limit_user_t(h, h->t2, h->w.vV64b, nullptr, gNe, -1.0, g + M);
}

// true residual r = g^N - n.D grad u^+ - rank-one term of the coupled
// u = v_V + v_B(psi) left by the refined solves (vV64 + u64, vV64b + u64b)
int true_residual_coupled_acc(kfbi_handle* h, const double* psi, const double* gNi, const double* gNe, double* r) {
  const int M = h->t.M;
  const double *xi, *xe;
  int rc;
  if ((rc = density_vector_buf(h, psi, h->w.xvec, &xi))) return rc;
  if ((rc = density_vector_buf(h, psi + M, h->w.xvec2, &xe))) return rc;
  if ((rc = launch_limit_user_t(h, h->t, h->w.vV64, nullptr, gNi, -1.0, r))) return rc;
  if ((rc = launch_limit_user_t(h, h->t, h->w.u64, xi, r, -1.0, r))) return rc;
  if ((rc = launch_limit_user_t(h, h->t2, h->w.vV64b, nullptr, gNe, -1.0, r + M))) return rc;
  if ((rc = launch_limit_user_t(h, h->t2, h->w.u64b, xe, r + M, -1.0, r + M))) return rc;
  return launch_rank_one_coupled(h, psi, r, -1.0);
}

// out = base + sgn * A psi    (A psi = dv_B^+/dn of the single layer)
int apply_A(kfbi_handle* h, int prec, double lambda, const double* psi, double* out, double sgn, const double* base) {
  if (h->coupled)
    return prec == KFBI_FP64 ? apply_A_coupled(h, lambda, psi, out, sgn, base)
                             : apply_A_coupled32(h, lambda, psi, out, sgn, base);
  const double* x;
  int rc = density_vector(h, psi, &x);
  if (rc) return rc;
  if ((rc = launch_correction(h, x, h->w.corr))) return rc;
  SolveArgs sa;
  sa.corr = h->w.corr;
  sa.lambda = lambda;
  if (prec == KFBI_FP64) {
    if ((rc = box_solve64(h, sa, h->w.grid64))) return rc;
    rc = launch_limit64(h, h->w.grid64, x, base, sgn, out);
  } else {
    if ((rc = box_solve32(h, sa, h->w.grid32))) return rc;
    rc = launch_limit32(h, h->w.grid32, x, base, sgn, out);
  }
  // Poisson case: A psi + <ds, psi>/|Gamma| (A alone is singular there)
  if (rc == KFBI_OK && lambda == 0.0) rc = launch_rank_one(h, psi, out, sgn);
  return rc;
}

// g = gN - dv_V^+/dn, v_V the box solve of alpha * src
int rhs_g(kfbi_handle* h, double lambda, const double* src, double alpha, const double* gN, double* g) {
  SolveArgs sa;
  sa.src = src;
  sa.alpha = alpha;
  sa.lambda = lambda;
  int rc = box_solve64(h, sa, h->w.grid64);
  if (rc) return rc;
  return launch_limit64(h, h->w.grid64, nullptr, gN, -1.0, g);
}

int read_scalar(kfbi_handle* h, const double* dev, double* out) {
  KFBI_CUDA(cudaMemcpyAsync(h->w.host_small, dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  KFBI_CUDA(cudaStreamSynchronize(h->stream));
  *out = h->w.host_small[0];
  return KFBI_OK;
}

// two device scalars with one synchronisation
int read_two(kfbi_handle* h, const double* a, const double* b, double* va, double* vb) {
  KFBI_CUDA(cudaMemcpyAsync(h->w.host_small, a, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  KFBI_CUDA(cudaMemcpyAsync(h->w.host_small + 1, b, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  KFBI_CUDA(cudaStreamSynchronize(h->stream));
  *va = h->w.host_small[0];
  *vb = h->w.host_small[1];
  return KFBI_OK;
}

int norm2(kfbi_handle* h, const double* v, double* slot, double* out) {
  int rc = vec_dots(h, v, 1, h->nk, v, slot);
  if (rc) return rc;
  double s;
  if ((rc = read_scalar(h, slot, &s))) return rc;
  *out = std::sqrt(s);
  return KFBI_OK;
}

// float64-accurate box solve from float32 transforms (iterative refinement
// with the float64 5/7-point residual): u = L_h^{-1}(alpha*src + corr) on the
// user layout.  Each round gains about -log10(kappa(L_h) eps_32) digits: one
// round leaves a relative error near 1e-12 at 256^3 and 1e-10 at 512^3, so
// GMRES tolerances below 1e-9 take a second round.
int refine_rounds(const kfbi_handle* h) { return h->opts.tol < 1e-9 ? 2 : 1; }

int refined_solve(kfbi_handle* h, const double* src, double alpha, const double* corr, double lambda, double* u) {
  // Dirichlet box, separate x and y passes: the first solve's float result
  // stays in the padded grid grid32 alone (no float64 copy), the correction
  // solve runs in grid32b and writes u = its result + grid32 in float64
  const bool split = h->grid.bc == KFBI_BOX_DIRICHLET && !(h->xy_fused && h->grid.dim == 3);
  SolveArgs sa;
  sa.src = src;
  sa.alpha = alpha;
  sa.corr = corr;
  sa.lambda = lambda;
  sa.out_user = split ? nullptr : u;
  int rc = box_solve32(h, sa, h->w.grid32);
  if (rc) return rc;
  const int rounds = refine_rounds(h);
  for (int r = 0; r < rounds; ++r) {
    SolveArgs sr;
    if (r == 0 && split) {
      // float-float residual of the float grid, float32 result; the
      // irregular nodes from the padded grid too
      if ((rc = launch_residual_ff(h, src, alpha, corr, h->w.grid32, nullptr, lambda, h->w.res32))) return rc;
      sr.src32 = h->w.res32;
      sr.lambda = lambda;
      sr.out_user = u;
      sr.aux32 = h->w.grid32;
      sr.keep = false;
      if ((rc = box_solve32(h, sr, h->w.grid32b))) return rc;
      continue;
    }
    if (r == 0) {
      // u is exactly the float32 grid of the solve just done: float-float
      // residual, float32 result
      if ((rc = launch_residual_ff(h, src, alpha, corr, h->w.grid32, u, lambda, h->w.res32))) return rc;
      sr.src32 = h->w.res32;
    } else {
      if ((rc = launch_residual(h, src, alpha, corr, u, lambda, h->w.res64))) return rc;
      sr.src = h->w.res64;
    }
    sr.lambda = lambda;
    sr.out_user = u;
    sr.aux = u;
    sr.beta = 1.0;
    sr.gamma = 1.0;
    sr.keep = false;  // only u is read after a refinement round
    if ((rc = box_solve32(h, sr, h->w.grid32))) return rc;
  }
  return KFBI_OK;
}

// out = base + sgn * A psi with a float64-accurate (refined) box solve
int apply_A_acc(kfbi_handle* h, double lambda, const double* psi, double* out, double sgn, const double* base) {
  if (h->coupled) return apply_A_acc_coupled(h, lambda, psi, out, sgn, base);
  const double* x;
  int rc = density_vector(h, psi, &x);
  if (rc) return rc;
  if ((rc = launch_correction(h, x, h->w.corr))) return rc;
  if ((rc = refined_solve(h, nullptr, 1.0, h->w.corr, lambda, h->w.u64))) return rc;
  if ((rc = launch_limit_user(h, h->w.u64, x, base, sgn, out))) return rc;
  return lambda == 0.0 ? launch_rank_one(h, psi, out, sgn) : KFBI_OK;
}

// g = gN - dv_V^+/dn with the refined volume solve (v_V kept in vV64)
int rhs_g_acc(kfbi_handle* h, double lambda, const double* src, double alpha, const double* gN, double* g) {
  int rc = refined_solve(h, src, alpha, nullptr, lambda, h->w.vV64);
  if (rc) return rc;
  return launch_limit_user(h, h->w.vV64, nullptr, gN, -1.0, g);
}

// Launches of one Arnoldi iteration (w = A v_j and the CGS2 step), all
// carrying the stop flag as their skip flag; the residual estimate and the
// device's stop decision go to the pinned host slots of iteration j.
struct SkipScope {
  kfbi_handle* h;
  SkipScope(kfbi_handle* hh, const int* flag) : h(hh) { h->skip = flag; }
  ~SkipScope() { h->skip = nullptr; }
};

int arnoldi_iteration(kfbi_handle* h, int prec, double lambda, int j, double gnorm, double tol) {
  const int M = h->nk, m = h->opts.restart;
  double* V = h->w.vecs;
  int rc;
  {
    SkipScope scope(h, h->w.stop);
    if ((rc = apply_A(h, prec, lambda, V + (size_t)j * M, h->w.tmp, 1.0, nullptr))) return rc;
    if ((rc = arnoldi_step(h, V, M, h->w.tmp, j, m, gnorm, tol))) return rc;
  }
  KFBI_CUDA(cudaMemcpyAsync(h->w.host_small + 128 + 2 * j, h->w.small + small_res(m), 2 * sizeof(double),
                            cudaMemcpyDeviceToHost, h->stream));
  KFBI_CUDA(cudaEventRecord(h->arn_ev[j & 1], h->stream));
  return KFBI_OK;
}

// GMRES(m) with CGS2 Arnoldi on A psi = g; psi in: initial guess, out: solution.
// zero_guess: psi is known to be zero, so the first residual is g itself.
// fallback (optional): an alternative initial guess whose squared residual
// norm ||g - A fallback||^2 is in the device slot fallback_res2; it replaces
// psi when psi's first residual is larger (both read with one
// synchronisation).
// gnorm_known (>= 0): ||g|| already read by the caller (saves a synchronisation).
int gmres(kfbi_handle* h, int prec, double lambda, const double* g, double* psi, kfbi_stats* st, double tol,
          int max_iter, bool zero_guess = false, const double* fallback = nullptr,
          const double* fallback_res2 = nullptr, double gnorm_known = -1.0) {
  const int M = h->nk;
  const int m = h->opts.restart;
  double* V = h->w.vecs;
  const int ld = M;
  double* r = h->w.r;
  double* s = h->w.small;
  int rc;
  double gnorm = gnorm_known;
  if (gnorm < 0.0 && (rc = norm2(h, g, s + small_nrm2(m), &gnorm))) return rc;
  const double gnorm_raw = gnorm;
  if (gnorm == 0.0) gnorm = 1.0;
  int it = 0;
  double rel = 0.0;
  bool first = true;
  for (;;) {
    if (first && zero_guess) {
      if ((rc = vec_copy(h, r, g, M))) return rc;
    } else if ((rc = apply_A(h, prec, lambda, psi, r, -1.0, g))) {  // r = g - A psi
      return rc;
    }
    if ((rc = vec_dots(h, r, 1, M, r, s + small_nrm2(m)))) return rc;
    double beta, fallback_res = 0.0;
    if (first && zero_guess) {
      beta = gnorm_raw;  // r = g: the same reduction as ||g||, no second read
    } else {
      double b2, f2 = 0.0;
      if (first && fallback != nullptr) {
        if ((rc = read_two(h, s + small_nrm2(m), fallback_res2, &b2, &f2))) return rc;
      } else if ((rc = read_scalar(h, s + small_nrm2(m), &b2))) {
        return rc;
      }
      beta = std::sqrt(b2);
      fallback_res = std::sqrt(f2);
    }
    if (first && fallback != nullptr && beta > fallback_res) {
      // the residual judges the guess: go back to the alternative
      if ((rc = vec_copy(h, psi, fallback, M))) return rc;
      fallback = nullptr;
      zero_guess = false;
      st->warmstart = 0;
      continue;
    }
    fallback = nullptr;
    rel = beta / gnorm;
    if (first) {
      st->init_rel_res = rel;
      first = false;
    }
    if (!std::isfinite(rel)) {
      set_error("non-finite residual in GMRES");
      return KFBI_ERR_NAN;
    }
    if (rel <= tol || it >= max_iter || beta == 0.0) break;
    if ((rc = launch_init_arnoldi(h, s, m))) return rc;
    if ((rc = vec_scale_by_norm(h, V, r, s + small_nrm2(m), M))) return rc;
    KFBI_CUDA(cudaMemsetAsync(h->w.stop, 0, sizeof(int), h->stream));
    // Iteration j + 1 is enqueued before the residual estimate of iteration
    // j reaches the host, so the device never waits for the host between
    // iterations; its launches do nothing when iteration j set the stop flag.
    if ((rc = arnoldi_iteration(h, prec, lambda, 0, gnorm, tol))) return rc;
    int jd = 0;
    for (int j = 0; j < m; ++j) {
      const bool ahead = j + 1 < m && it + 2 <= max_iter;
      if (ahead && (rc = arnoldi_iteration(h, prec, lambda, j + 1, gnorm, tol))) return rc;
      KFBI_CUDA(cudaEventSynchronize(h->arn_ev[j & 1]));
      const double res = h->w.host_small[128 + 2 * j];
      const bool stop = h->w.host_small[128 + 2 * j + 1] != 0.0;
      ++it;
      rel = res / gnorm;
      jd = j + 1;
      if (!std::isfinite(rel)) {
        set_error("non-finite residual in GMRES");
        return KFBI_ERR_NAN;
      }
      if (stop || rel <= tol || it >= max_iter || !ahead) break;
    }
    if ((rc = arnoldi_solve(h, s, jd, m))) return rc;
    if ((rc = vec_update(h, psi, V, jd, ld, s + small_y(m), 1.0))) return rc;
    if (rel <= tol || it >= max_iter) break;
  }
  st->iters = it;
  st->rel_res = rel;
  return rel <= tol ? KFBI_OK : KFBI_ERR_NOT_CONVERGED;
}

int richardson(kfbi_handle* h, int prec, double lambda, const double* g, double* psi, kfbi_stats* st) {
  const int M = h->nk;
  double* r = h->w.r;
  double* s = h->w.small;
  const int m = h->opts.restart;
  int rc;
  double gnorm;
  if ((rc = norm2(h, g, s + small_nrm2(m), &gnorm))) return rc;
  if (gnorm == 0.0) gnorm = 1.0;
  int it = 0;
  double rel = 0.0;
  for (;;) {
    // float32 transforms: float64-accurate residuals (refined solves), so
    // the iteration reaches float64 tolerances
    rc = prec == KFBI_FP64 ? apply_A(h, prec, lambda, psi, r, -1.0, g) : apply_A_acc(h, lambda, psi, r, -1.0, g);
    if (rc) return rc;
    double rn;
    if ((rc = norm2(h, r, s + small_nrm2(m), &rn))) return rc;
    rel = rn / gnorm;
    if (it == 0) st->init_rel_res = rel;
    if (!std::isfinite(rel)) {
      set_error("non-finite residual in the simple iteration");
      return KFBI_ERR_NAN;
    }
    if (rel <= h->opts.tol || it >= h->opts.max_iter) break;
    if ((rc = vec_axpby(h, psi, 2.0 * h->opts.gamma, r, 1.0, M))) return rc;
    ++it;
  }
  st->iters = it;
  st->rel_res = rel;
  return rel <= h->opts.tol ? KFBI_OK : KFBI_ERR_NOT_CONVERGED;
}

// GMRES with iterative refinement (Carson and Higham): the outer residual
// r = g - A psi uses float64-accurate box solves, the inner correction solve
// A delta = r runs GMRES with float32 box solves and float64 Arnoldi.
// fallback (optional): an alternative initial guess whose squared residual
// norm is in the device slot fallback_res2; it replaces psi when psi's first
// residual is larger.  gnorm_known (>= 0): ||g|| already read by the caller.
// rF (optional, with fallback): the fallback's residual vector g - A fallback
// to float64 accuracy.  psi's first residual is then rF - A (psi - fallback)
// with float32 transforms: the difference is small (of the order of rF), so
// the float32 operator's relative error of ~1e-6 enters at ~1e-6 ||rF||, far
// below the tolerance, and the first refined solve is saved.
int gmres_ir(kfbi_handle* h, double lambda, const double* g, double* psi, kfbi_stats* st,
             const double* fallback = nullptr, const double* fallback_res2 = nullptr, double gnorm_known = -1.0,
             const double* rF = nullptr) {
  const int M = h->nk;
  double* r = h->w.r2;
  double* delta = h->w.tmp2;
  double* slot = h->w.small + small_nrm2(h->opts.restart);
  const double tol = h->opts.tol;
  int rc;
  double gnorm = gnorm_known;
  if (gnorm < 0.0 && (rc = norm2(h, g, slot, &gnorm))) return rc;
  if (gnorm == 0.0) gnorm = 1.0;
  int inner_total = 0, outer = 0;
  double rel = 0.0;
  bool approx = false;  // rn came from the residual by difference
  for (;;) {
    double rn, fallback_res = 0.0;
    if (outer == 0 && fallback != nullptr && rF != nullptr) {
      approx = true;
      // residual by difference (no refined solve); the residual judges the
      // guess, and the fallback's residual is rF itself
      double rn2, f2;
      if ((rc = vec_copy(h, delta, psi, M))) return rc;
      if ((rc = vec_axpby(h, delta, -1.0, fallback, 1.0, M))) return rc;
      if ((rc = apply_A(h, KFBI_MIXED, lambda, delta, r, -1.0, rF))) return rc;
      if ((rc = vec_dots(h, r, 1, M, r, slot))) return rc;
      if ((rc = read_two(h, slot, fallback_res2, &rn2, &f2))) return rc;
      rn = std::sqrt(rn2);
      fallback_res = std::sqrt(f2);
      if (rn > fallback_res) {
        if ((rc = vec_copy(h, psi, fallback, M))) return rc;
        if ((rc = vec_copy(h, r, rF, M))) return rc;
        rn = fallback_res;
        st->warmstart = 0;
      }
      fallback = nullptr;
    } else if ((rc = apply_A_acc(h, lambda, psi, r, -1.0, g))) {
      return rc;
    } else if (outer == 0 && fallback != nullptr) {
      double rn2, f2;
      if ((rc = vec_dots(h, r, 1, M, r, slot))) return rc;
      if ((rc = read_two(h, slot, fallback_res2, &rn2, &f2))) return rc;
      rn = std::sqrt(rn2);
      fallback_res = std::sqrt(f2);
    } else if ((rc = norm2(h, r, slot, &rn))) {
      return rc;
    }
    if (outer == 0 && fallback != nullptr && rn > fallback_res) {
      // the residual judges the guess: go back to the alternative
      if ((rc = vec_copy(h, psi, fallback, M))) return rc;
      fallback = nullptr;
      st->warmstart = 0;
      continue;
    }
    fallback = nullptr;
    rel = rn / gnorm;
    if (outer == 0) st->init_rel_res = rel;
    if (!std::isfinite(rel)) {
      set_error("non-finite residual in GMRES-IR");
      return KFBI_ERR_NAN;
    }
    if (rel <= tol || inner_total >= h->opts.max_iter || outer >= 20) {
      // the solver stops on a float64-accurate residual only (it also
      // leaves v_B(psi) in u64 for the caller)
      if (!approx) break;
      approx = false;
      rF = nullptr;
      continue;
    }
    approx = false;
    // inner tolerance relative to ||r||: as far as the float32 operator can
    // go (six digits), or what the target needs with a factor of 1.25 to
    // spare (the inner solve overshoots its target, and the float32
    // operator adds ~1e-5 ||r|| to the next outer residual).  Measured on the
    // 256^3 prolate shell (steps 6-25): factors 0.1 / 0.25 / 0.5 / 0.8 / 1.0 gave 11.8 /
    // 10.6 / 9.8 / 9.25 / 9.2 inner iterations and 1.25 / 1.25 / 1.25 / 1.3
    // / 1.35 outer rounds per step, 0.8 the shortest step.
    double tin = std::max(1e-6, 0.8 * tol * gnorm / rn);
    if (tin > 0.5) tin = 0.5;
    KFBI_CUDA(cudaMemsetAsync(delta, 0, sizeof(double) * (size_t)M, h->stream));
    kfbi_stats in{};
    rc = gmres(h, KFBI_MIXED, lambda, r, delta, &in, tin, h->opts.max_iter - inner_total, true, nullptr, nullptr, rn);
    if (rc != KFBI_OK && rc != KFBI_ERR_NOT_CONVERGED) return rc;
    inner_total += in.iters;
    if ((rc = vec_axpby(h, psi, 1.0, delta, 1.0, M))) return rc;
    ++outer;
  }
  st->iters = inner_total;
  st->outer = outer;
  st->rel_res = rel;
  return rel <= tol ? KFBI_OK : KFBI_ERR_NOT_CONVERGED;
}

int solve_bie(kfbi_handle* h, int prec, double lambda, const double* g, double* psi, kfbi_stats* st,
              const double* fallback = nullptr, const double* fallback_res2 = nullptr, double gnorm_known = -1.0,
              const double* rF = nullptr) {
  if (h->opts.solver == KFBI_RICHARDSON) return richardson(h, prec, lambda, g, psi, st);
  if (prec != KFBI_FP64) return gmres_ir(h, lambda, g, psi, st, fallback, fallback_res2, gnorm_known, rF);
  return gmres(h, prec, lambda, g, psi, st, h->opts.tol, h->opts.max_iter, false, fallback, fallback_res2,
               gnorm_known);
}

// ------------------------------------------------ projection warm start
// The densities psi_s of earlier solves and their right-hand sides g_s
// satisfy A psi_s = g_s to the solver tolerance, so for any coefficients c
// the residual of psi_F = sum c_s psi_s is g - sum c_s g_s without applying
// A.  c minimises that residual (normal equations of the k <= KFBI_HISTORY
// stored g_s, Cholesky on the host, columns that are numerically dependent
// on earlier ones dropped).
// out: gnorm = ||g||; rF2 = the device slot that receives ||r_F||^2 (read
// by the solver together with its first residual).  One synchronisation.
int project_history(kfbi_handle* h, const double* g, double* gnorm, const double** rF2) {
  const int M = h->nk;
  const int k = h->hist_count < KFBI_HISTORY ? h->hist_count : KFBI_HISTORY;
  double* G = h->w.proj;             // [k][k]
  double* b = G + KFBI_HISTORY * KFBI_HISTORY;
  double* cdev = b + KFBI_HISTORY;
  double* sq = cdev + KFBI_HISTORY;  // ||psi_F||^2 (learned form), ||r_F||^2, ||g||^2
  int rc;
  if ((rc = vec_copy(h, h->w.rF, g, M))) return rc;
  KFBI_CUDA(cudaMemsetAsync(h->w.psiF, 0, sizeof(double) * (size_t)M, h->stream));
  if ((rc = launch_gram(h, h->w.hist_g, k, g, G, b, sq + 2))) return rc;
  double* hs = h->w.host_small;
  const int nread = KFBI_HISTORY * (KFBI_HISTORY + 2) + 3;
  KFBI_CUDA(cudaMemcpyAsync(hs, G, sizeof(double) * (size_t)nread, cudaMemcpyDeviceToHost, h->stream));
  KFBI_CUDA(cudaStreamSynchronize(h->stream));
  *gnorm = std::sqrt(hs[nread - 1]);
  if (k > 0) {
    double A[KFBI_HISTORY][KFBI_HISTORY], L[KFBI_HISTORY][KFBI_HISTORY] = {}, y[KFBI_HISTORY] = {},
                                          c[KFBI_HISTORY] = {}, rhs[KFBI_HISTORY];
    bool keep[KFBI_HISTORY];
    double dmax = 0.0;
    for (int i = 0; i < k; ++i) {
      for (int j = 0; j < k; ++j) A[i][j] = hs[i * k + j];
      rhs[i] = hs[KFBI_HISTORY * KFBI_HISTORY + i];
      dmax = std::max(dmax, A[i][i]);
    }
    // Cholesky with dependent columns skipped
    for (int j = 0; j < k; ++j) {
      double d = A[j][j];
      for (int p = 0; p < j; ++p)
        if (keep[p]) d -= L[j][p] * L[j][p];
      keep[j] = d > 1e-13 * dmax && dmax > 0.0;
      if (!keep[j]) continue;
      L[j][j] = std::sqrt(d);
      for (int i = j + 1; i < k; ++i) {
        double v = A[i][j];
        for (int p = 0; p < j; ++p)
          if (keep[p]) v -= L[i][p] * L[j][p];
        L[i][j] = v / L[j][j];
      }
    }
    for (int i = 0; i < k; ++i) {
      if (!keep[i]) continue;
      double v = rhs[i];
      for (int p = 0; p < i; ++p)
        if (keep[p]) v -= L[i][p] * y[p];
      y[i] = v / L[i][i];
    }
    for (int i = k - 1; i >= 0; --i) {
      if (!keep[i]) continue;
      double v = y[i];
      for (int p = i + 1; p < k; ++p)
        if (keep[p]) v -= L[p][i] * c[p];
      c[i] = v / L[i][i];
    }
    for (int i = 0; i < k; ++i) hs[i] = c[i];
    KFBI_CUDA(cudaMemcpyAsync(cdev, hs, sizeof(double) * (size_t)k, cudaMemcpyHostToDevice, h->stream));
    if ((rc = vec_update(h, h->w.psiF, h->w.hist_psi, k, M, cdev, 1.0))) return rc;
    if ((rc = vec_update(h, h->w.rF, h->w.hist_g, k, M, cdev, -1.0))) return rc;
  }
  if ((rc = vec_dots(h, h->w.rF, 1, M, h->w.rF, sq + 1))) return rc;
  *rF2 = sq + 1;
  return KFBI_OK;
}

// stores psi and its image A psi: g - r with r = g - A psi the solver's
// final float64-accurate residual when given, else g (A psi to the tolerance)
int push_history(kfbi_handle* h, const double* psi, const double* g, const double* r = nullptr) {
  const int M = h->nk;
  const size_t slot = (size_t)(h->hist_count % KFBI_HISTORY) * M;
  int rc;
  if ((rc = vec_copy(h, h->w.hist_psi + slot, psi, M))) return rc;
  if ((rc = vec_copy(h, h->w.hist_g + slot, g, M))) return rc;
  if (r != nullptr && (rc = vec_axpby(h, h->w.hist_g + slot, -1.0, r, 1.0, M))) return rc;
  ++h->hist_count;
  return KFBI_OK;
}

int check_handle(kfbi_handle* h) {
  if (h == nullptr) {
    kfbi::set_error("null handle");
    return KFBI_ERR_ARG;
  }
  return KFBI_OK;
}

double elapsed_ms(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace kfbi

using namespace kfbi;

extern "C" {

const char* kfbi_last_error(void) { return kfbi::g_err; }

static int create_impl(const kfbi_geometry* geom, const kfbi_grid* grid, double sigma_i, double sigma_e, double dt,
                       const kfbi_opts* opts, kfbi_handle** out, const double* D_i, const double* D_e);

int kfbi_create(const kfbi_geometry* geom, const kfbi_grid* grid, double sigma_i, double sigma_e, double dt,
                const kfbi_opts* opts, kfbi_handle** out) {
  return create_impl(geom, grid, sigma_i, sigma_e, dt, opts, out, nullptr, nullptr);
}

int kfbi_create_coupled(const kfbi_geometry* geom, const kfbi_grid* grid, const double* D_i, const double* D_e,
                        double dt, const kfbi_opts* opts, kfbi_handle** out) {
  if (!D_i || !D_e || !grid) {
    set_error("null conductivities");
    return KFBI_ERR_ARG;
  }
  for (int a = 0; a < grid->dim && a < 3; ++a)
    if (!(D_i[a] > 0.0) || !(D_e[a] > 0.0)) {
      set_error("conductivities must be positive");
      return KFBI_ERR_ARG;
    }
  if (opts && opts->precision != KFBI_FP64 && opts->precision != KFBI_MIXED) {
    set_error("the coupled system is solved in float64 (KFBI_FP64) or with float32 transforms (KFBI_MIXED)");
    return KFBI_ERR_ARG;
  }
  if (grid->box != KFBI_BOX_DIRICHLET) {
    set_error("the coupled system is solved in the Dirichlet box");
    return KFBI_ERR_ARG;
  }
  return create_impl(geom, grid, D_i[0], D_e[0], dt, opts, out, D_i, D_e);
}

static int create_impl(const kfbi_geometry* geom, const kfbi_grid* grid, double sigma_i, double sigma_e, double dt,
                       const kfbi_opts* opts, kfbi_handle** out, const double* D_i, const double* D_e) {
  if (!geom || !grid || !out || !opts) {
    set_error("null argument");
    return KFBI_ERR_ARG;
  }
  *out = nullptr;
  if (grid->dim != 2 && grid->dim != 3) {
    set_error("dim must be 2 or 3");
    return KFBI_ERR_ARG;
  }
  if (geom->dim != grid->dim || !dst_supported(grid->N) || (grid->dim == 2 && grid->N < 16)) {
    set_error("unsupported grid: N=%d dim=%d (N in 8,16,32,64,128,256,384,512; 2-D needs N >= 16)", grid->N,
              grid->dim);
    return KFBI_ERR_ARG;
  }
  if (geom->n_nodes < 8 || geom->nodes == nullptr || !(grid->hi > grid->lo)) {
    set_error("bad geometry or grid extents");
    return KFBI_ERR_ARG;
  }
  if (grid->dim == 3 && geom->kind == KFBI_MESH3) {
    if (geom->tri == nullptr || geom->n_tri <= 0) {
      set_error("a mesh domain needs its triangles");
      return KFBI_ERR_ARG;
    }
  } else if (grid->dim == 3 && (geom->tri == nullptr || geom->n_tri <= 0 || geom->cube_t == nullptr ||
                                geom->n_comp < 1 || geom->n_comp > KFBI_MAX_COMP)) {
    set_error("3-D geometry needs a triangle mesh and cube-sphere tables");
    return KFBI_ERR_ARG;
  }
  if (opts->restart < 1 || opts->restart > MAX_RESTART || !(sigma_i > 0) || !(sigma_e > 0) || !(dt > 0)) {
    set_error("bad options (restart in 1..%d, positive conductivities and dt)", MAX_RESTART);
    return KFBI_ERR_ARG;
  }
  if (grid->box != KFBI_BOX_DIRICHLET && grid->box != KFBI_BOX_NEUMANN) {
    set_error("box must be KFBI_BOX_DIRICHLET or KFBI_BOX_NEUMANN");
    return KFBI_ERR_ARG;
  }

  kfbi_handle* h = new kfbi_handle();
  h->opts = *opts;
  h->stream = (cudaStream_t)opts->stream;
  h->sigma_i = sigma_i;
  h->sigma_e = sigma_e;
  h->dt = dt;
  h->lambda = (2.0 / dt) * (1.0 / sigma_i + 1.0 / sigma_e);
  if (D_i != nullptr) {
    h->coupled = true;
    for (int a = 0; a < 3; ++a) {
      h->cpl.di[a] = a < grid->dim ? D_i[a] : 1.0;
      h->cpl.de[a] = a < grid->dim ? D_e[a] : 1.0;
    }
    h->cpl.kappa = 2.0 / dt;  // Cm beta / (dt/2) with Cm beta = 1
  }
  GeomParams& gp = h->gp;
  memset(&gp, 0, sizeof(gp));
  gp.dim = geom->dim;
  gp.kind = geom->kind;
  gp.n_comp = grid->dim == 3 && geom->kind != KFBI_MESH3 ? geom->n_comp : 1;
  for (int i = 0; i < 16; ++i) gp.p[i] = geom->params[i];
  for (int c = 0; c < KFBI_MAX_COMP && geom->kind != KFBI_MESH3; ++c) {
    gp.comp_map[c] = geom->comp_map[c];
    for (int k = 0; k < 3; ++k) gp.comp_axes[c][k] = geom->comp_axes[c][k];
    gp.comp_tri_offset[c] = geom->comp_tri_offset[c];
    gp.comp_vert_offset[c] = geom->comp_vert_offset[c];
  }
  gp.cube_n = geom->cube_n;
  h->grid.dim = grid->dim;
  h->grid.N = grid->N;
  h->grid.lo = grid->lo;
  h->grid.h = (grid->hi - grid->lo) / grid->N;
  h->grid.bc = grid->box;
  h->rinv_ok = true;
  int rc;
  auto fail = [&](int code) {
    kfbi_destroy(h);
    return code;
  };
  if ((rc = dalloc(h, &h->w.err, 4))) return fail(rc);
  if ((rc = dalloc(h, &h->w.stop, 4))) return fail(rc);
  if ((rc = dalloc(h, &h->w.counter, 4))) return fail(rc);
  if (cudaMemsetAsync(h->w.stop, 0, 4 * sizeof(int), h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->w.counter, 0, 4 * sizeof(unsigned), h->stream) != cudaSuccess) {
    set_error("cudaMemset failed");
    return fail(KFBI_ERR_CUDA);
  }
  for (cudaEvent_t& e : h->arn_ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      set_error("cudaEventCreate failed");
      return fail(KFBI_ERR_CUDA);
    }
  if ((rc = setup_build(h, geom))) return fail(rc);
  const int m = opts->restart;
  // Krylov vectors, densities and their history: M entries, 2M for the
  // coupled system's density pair
  h->nk = h->coupled ? 2 * h->t.M : h->t.M;
  const int M = h->nk;
  const int64_t P = padded_points(h);
  if ((rc = dalloc(h, &h->w.grid64, (size_t)P))) return fail(rc);
  if ((rc = dalloc(h, &h->w.grid32, (size_t)P))) return fail(rc);
  // the second float grid: the extracellular field of coupled solves, the
  // correction solve of a refined scalar solve (the first solve's float
  // result stays in grid32)
  if ((rc = dalloc(h, &h->w.grid32b, (size_t)P))) return fail(rc);
  if (cudaMemsetAsync(h->w.grid64, 0, sizeof(double) * (size_t)P, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->w.grid32, 0, sizeof(float) * (size_t)P, h->stream) != cudaSuccess ||
      cudaMemsetAsync(h->w.grid32b, 0, sizeof(float) * (size_t)P, h->stream) != cudaSuccess) {
    set_error("cudaMemset failed");
    return fail(KFBI_ERR_CUDA);
  }
  if ((rc = make_tma_maps(h))) return fail(rc);
  if ((rc = dalloc(h, &h->w.corr, (size_t)h->t.n_irr))) return fail(rc);
  if ((rc = dalloc(h, &h->w.xvec, (size_t)2 * h->t.M))) return fail(rc);
  if (h->coupled) {
    if ((rc = dalloc(h, &h->w.corr2, (size_t)h->t.n_irr))) return fail(rc);
    if ((rc = dalloc(h, &h->w.xvec2, (size_t)2 * h->t.M))) return fail(rc);
    if ((rc = dalloc(h, &h->w.grid64b, (size_t)P))) return fail(rc);
    if (cudaMemsetAsync(h->w.grid64b, 0, sizeof(double) * (size_t)P, h->stream) != cudaSuccess) {
      set_error("cudaMemset failed");
      return fail(KFBI_ERR_CUDA);
    }
    for (double** p : {&h->w.u64b, &h->w.vV64b, &h->w.res64b})
      if ((rc = dalloc(h, p, (size_t)grid_points(h)))) return fail(rc);
    if ((rc = dalloc(h, &h->w.res32b, (size_t)grid_points(h)))) return fail(rc);
  }
  if ((rc = dalloc(h, &h->w.vecs, (size_t)(m + 1) * M))) return fail(rc);
  if ((rc = dalloc(h, &h->w.small, (size_t)small_size(MAX_RESTART)))) return fail(rc);
  if ((rc = dalloc(h, &h->w.partial, (size_t)KFBI_ARN_BLOCKS * (MAX_RESTART + 2) + 16))) return fail(rc);
  if ((rc = dalloc(h, &h->w.g, (size_t)M))) return fail(rc);
  if ((rc = dalloc(h, &h->w.r, (size_t)M))) return fail(rc);
  if ((rc = dalloc(h, &h->w.tmp, (size_t)M))) return fail(rc);
  if ((rc = dalloc(h, &h->w.tmp2, (size_t)M))) return fail(rc);
  if ((rc = dalloc(h, &h->w.psi_prev, (size_t)M))) return fail(rc);
  if ((rc = dalloc(h, &h->w.r2, (size_t)M))) return fail(rc);
  if ((rc = dalloc(h, &h->w.psi_prev2, (size_t)M))) return fail(rc);
  if ((rc = dalloc(h, &h->w.psi_save, (size_t)M))) return fail(rc);
  if ((rc = dalloc(h, &h->w.psi_learn, (size_t)M))) return fail(rc);
  if ((rc = dalloc(h, &h->w.g_prev, (size_t)M))) return fail(rc);
  cudaMemsetAsync(h->w.g_prev, 0, sizeof(double) * (size_t)M, h->stream);
  cudaMemsetAsync(h->w.psi_prev2, 0, sizeof(double) * (size_t)M, h->stream);
  if ((rc = dalloc(h, &h->w.u64, (size_t)grid_points(h)))) return fail(rc);
  if ((rc = dalloc(h, &h->w.res64, (size_t)grid_points(h)))) return fail(rc);
  if ((rc = dalloc(h, &h->w.res32, (size_t)grid_points(h)))) return fail(rc);
  if ((rc = dalloc(h, &h->w.vV64, (size_t)grid_points(h)))) return fail(rc);
  cudaMemsetAsync(h->w.psi_prev, 0, sizeof(double) * (size_t)M, h->stream);
  if ((rc = dalloc(h, &h->w.hist_psi, (size_t)KFBI_HISTORY * M))) return fail(rc);
  if ((rc = dalloc(h, &h->w.hist_g, (size_t)KFBI_HISTORY * M))) return fail(rc);
  if ((rc = dalloc(h, &h->w.psiF, (size_t)M))) return fail(rc);
  if ((rc = dalloc(h, &h->w.rF, (size_t)M))) return fail(rc);
  if ((rc = dalloc(h, &h->w.proj, (size_t)KFBI_HISTORY * (KFBI_HISTORY + 2) + 8))) return fail(rc);
  // [0, 128): scalars and the projection system (which may run past 128 for
  // long histories: it is read before GMRES starts); [128, 128 + 2
  // MAX_RESTART): per-iteration residual estimates and stop flags of GMRES
  constexpr int host_small_n = std::max(128 + 2 * MAX_RESTART, KFBI_HISTORY * (KFBI_HISTORY + 2) + 3);
  if (cudaMallocHost((void**)&h->w.host_small, host_small_n * sizeof(double)) != cudaSuccess) {
    set_error("cudaMallocHost failed");
    return fail(KFBI_ERR_OOM);
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    set_error("setup failed: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(KFBI_ERR_CUDA);
  }
  *out = h;
  return KFBI_OK;
}

void kfbi_destroy(kfbi_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  for (void* p : h->allocations) cudaFree(p);
  if (h->w.host_small) cudaFreeHost(h->w.host_small);
  for (cudaEvent_t e : h->arn_ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->step_events) cudaEventDestroy(e);
  if (h->w.step_sq) cudaFree(h->w.step_sq);
  delete h;
}

int kfbi_query(kfbi_handle* h, kfbi_info* info) {
  if (int rc = check_handle(h)) return rc;
  if (!info) {
    set_error("null info");
    return KFBI_ERR_ARG;
  }
  info->M = h->t.M;
  info->n_irregular = h->t.n_irr;
  info->n_crossings = h->t.n_int;
  info->n_inside = h->t.n_inside;
  info->device_bytes = h->device_bytes;
  info->lambda = h->lambda;
  info->xy_fused = h->xy_fused ? 1 : 0;
  return KFBI_OK;
}

int kfbi_set_opts(kfbi_handle* h, const kfbi_opts* opts) {
  if (int rc = check_handle(h)) return rc;
  if (!opts || opts->restart < 1 || opts->restart > MAX_RESTART) {
    set_error("bad options");
    return KFBI_ERR_ARG;
  }
  if (opts->restart > h->opts.restart) {
    set_error("restart cannot grow after kfbi_create");
    return KFBI_ERR_ARG;
  }

  h->opts = *opts;
  h->stream = (cudaStream_t)opts->stream;
  return KFBI_OK;
}

int kfbi_export_setup(kfbi_handle* h, uint8_t* inside, int32_t* irregular, int32_t* crossing_axis,
                      int32_t* crossing_lo, double* crossing_z, int32_t* center, int8_t* sign) {
  if (int rc = check_handle(h)) return rc;
  const Tables& t = h->t;
  const int d = h->grid.dim;
  cudaStream_t st = h->stream;
  if (inside) KFBI_CUDA(cudaMemcpyAsync(inside, t.inside, (size_t)interior_points(h), cudaMemcpyDeviceToHost, st));
  if (irregular) KFBI_CUDA(cudaMemcpyAsync(irregular, t.irr, sizeof(int32_t) * t.n_irr, cudaMemcpyDeviceToHost, st));
  if (crossing_axis)
    KFBI_CUDA(cudaMemcpyAsync(crossing_axis, t.c_axis, sizeof(int32_t) * t.n_int, cudaMemcpyDeviceToHost, st));
  if (crossing_lo) KFBI_CUDA(cudaMemcpyAsync(crossing_lo, t.c_lo, sizeof(int32_t) * t.n_int, cudaMemcpyDeviceToHost, st));
  if (crossing_z) KFBI_CUDA(cudaMemcpyAsync(crossing_z, t.c_z, sizeof(double) * t.n_int, cudaMemcpyDeviceToHost, st));
  if (center) KFBI_CUDA(cudaMemcpyAsync(center, t.n_center, sizeof(int32_t) * t.M * d, cudaMemcpyDeviceToHost, st));
  if (sign) KFBI_CUDA(cudaMemcpyAsync(sign, t.n_sign, sizeof(int8_t) * t.M * d, cudaMemcpyDeviceToHost, st));
  KFBI_CUDA(cudaStreamSynchronize(st));
  return KFBI_OK;
}

int kfbi_export_tables(kfbi_handle* h, double* node_wn, int32_t* node_cnt, int32_t* node_pid, double* node_w,
                       int32_t* cross_cnt, int32_t* cross_pid, double* cross_wlo, double* cross_whi) {
  if (int rc = check_handle(h)) return rc;
  const Tables& t = h->t;
  cudaStream_t st = h->stream;
  const size_t M = t.M, NI = t.n_int, R = PATCH_MAX + 1;
  if (node_wn) KFBI_CUDA(cudaMemcpyAsync(node_wn, t.n_wn, sizeof(double) * M * t.P, cudaMemcpyDeviceToHost, st));
  if (node_cnt) KFBI_CUDA(cudaMemcpyAsync(node_cnt, t.n_dcnt, sizeof(int32_t) * M, cudaMemcpyDeviceToHost, st));
  if (node_pid) KFBI_CUDA(cudaMemcpyAsync(node_pid, t.n_dpid, sizeof(int32_t) * M * R, cudaMemcpyDeviceToHost, st));
  if (node_w) KFBI_CUDA(cudaMemcpyAsync(node_w, t.n_dw, sizeof(double) * M * R, cudaMemcpyDeviceToHost, st));
  if (cross_cnt) KFBI_CUDA(cudaMemcpyAsync(cross_cnt, t.c_cnt, sizeof(int32_t) * NI, cudaMemcpyDeviceToHost, st));
  if (cross_pid)
    KFBI_CUDA(cudaMemcpyAsync(cross_pid, t.c_pid, sizeof(int32_t) * NI * PATCH_MAX, cudaMemcpyDeviceToHost, st));
  if (cross_wlo)
    KFBI_CUDA(cudaMemcpyAsync(cross_wlo, t.c_wlo, sizeof(double) * NI * PATCH_MAX, cudaMemcpyDeviceToHost, st));
  if (cross_whi)
    KFBI_CUDA(cudaMemcpyAsync(cross_whi, t.c_whi, sizeof(double) * NI * PATCH_MAX, cudaMemcpyDeviceToHost, st));
  KFBI_CUDA(cudaStreamSynchronize(st));
  return KFBI_OK;
}

int kfbi_box_solve(kfbi_handle* h, int precision, double lambda, const double* r_dev, double* v_dev) {
  if (int rc = check_handle(h)) return rc;
  if (!r_dev || !v_dev) {
    set_error("null field");
    return KFBI_ERR_ARG;
  }

  SolveArgs sa;
  sa.src = r_dev;
  sa.lambda = lambda;
  sa.out_user = v_dev;
  if (precision == KFBI_FP64) return box_solve64(h, sa, h->w.grid64);
  if (precision == KFBI_MIXED || precision == KFBI_MIXED_LEARNED)
    return refined_solve(h, r_dev, 1.0, nullptr, lambda, v_dev);
  return box_solve32(h, sa, h->w.grid32);
}

int kfbi_correction(kfbi_handle* h, const double* psi_dev, double* rhs_dev) {
  if (int rc = check_handle(h)) return rc;
  const double* x;
  int rc = density_vector(h, psi_dev, &x);
  if (rc) return rc;
  if ((rc = launch_correction(h, x, h->w.corr))) return rc;
  return launch_scatter_grid(h, h->w.corr, rhs_dev);
}

int kfbi_interface_limit(kfbi_handle* h, const double* v_dev, const double* psi_dev, double* out_dev) {
  if (int rc = check_handle(h)) return rc;
  // place v in the padded grid (x passes of a zero-lambda identity are not
  // needed: copy through a solve-free scatter)
  int rc;
  const double* x = nullptr;
  if (psi_dev) {
    if ((rc = density_vector(h, psi_dev, &x))) return rc;
  }
  const int N = h->grid.N, n1 = N - 1;
  // user -> padded copy (rows of n1 values into rows of N); the Neumann box's
  // work grid has the field layout
  if (neumann_box(h)) {
    KFBI_CUDA(cudaMemcpyAsync(h->w.grid64, v_dev, sizeof(double) * (size_t)grid_points(h), cudaMemcpyDeviceToDevice,
                              h->stream));
  } else if (h->grid.dim == 3) {
    cudaMemcpy3DParms prm = {};
    prm.srcPtr = make_cudaPitchedPtr((void*)v_dev, sizeof(double) * n1, n1, n1);
    prm.dstPtr = make_cudaPitchedPtr((void*)h->w.grid64, sizeof(double) * N, N, N);
    prm.dstPos = make_cudaPos(sizeof(double), 1, 1);
    prm.extent = make_cudaExtent(sizeof(double) * n1, n1, n1);
    prm.kind = cudaMemcpyDeviceToDevice;
    KFBI_CUDA(cudaMemcpy3DAsync(&prm, h->stream));
  } else {
    KFBI_CUDA(cudaMemcpy2DAsync(h->w.grid64 + N + 1, sizeof(double) * N, v_dev, sizeof(double) * n1,
                                sizeof(double) * n1, n1, cudaMemcpyDeviceToDevice, h->stream));
  }
  return launch_limit64(h, h->w.grid64, x, nullptr, 1.0, out_dev);
}

int kfbi_apply_A(kfbi_handle* h, int precision, double lambda, const double* psi_dev, double* out_dev) {
  if (int rc = check_handle(h)) return rc;
  return apply_A(h, precision, lambda, psi_dev, out_dev, 1.0, nullptr);
}

int kfbi_rhs_g(kfbi_handle* h, double lambda, const double* f_dev, const double* gN_dev, double* g_dev) {
  if (int rc = check_handle(h)) return rc;
  return rhs_g(h, lambda, f_dev, 1.0, gN_dev, g_dev);
}

int kfbi_solve_bie(kfbi_handle* h, double lambda, const double* g_dev, double* psi_dev, kfbi_stats* stats) {
  if (int rc = check_handle(h)) return rc;
  kfbi_stats st{};
  auto t0 = std::chrono::steady_clock::now();
  int rc = solve_bie(h, KFBI_FP64, lambda, g_dev, psi_dev, &st);
  st.ms = elapsed_ms(t0);
  st.true_rel_res = -1.0;
  if (stats) *stats = st;
  return rc;
}

int kfbi_solve_neumann(kfbi_handle* h, double lambda, const double* f_dev, const double* gN_dev, double* u_dev,
                       double* psi_dev, kfbi_stats* stats) {
  if (int rc = check_handle(h)) return rc;
  if (!f_dev || !gN_dev || !u_dev || !psi_dev) {
    set_error("null argument");
    return KFBI_ERR_ARG;
  }
  if (h->coupled) {
    set_error("a coupled handle solves the vector problem: kfbi_solve_coupled");
    return KFBI_ERR_ARG;
  }
  kfbi_stats st{};
  auto t0 = std::chrono::steady_clock::now();
  const int prec = h->opts.precision == KFBI_FP64 ? KFBI_FP64 : KFBI_MIXED;
  int rc = prec == KFBI_FP64 ? rhs_g(h, lambda, f_dev, 1.0, gN_dev, h->w.g)
                             : rhs_g_acc(h, lambda, f_dev, 1.0, gN_dev, h->w.g);
  if (rc) return rc;
  const int solve_rc = solve_bie(h, prec, lambda, h->w.g, psi_dev, &st);
  if (solve_rc != KFBI_OK && solve_rc != KFBI_ERR_NOT_CONVERGED) return solve_rc;
  // u = v_V + v_B(psi) in one solve of the combined right-hand side
  const double* x;
  if ((rc = density_vector(h, psi_dev, &x))) return rc;
  if ((rc = launch_correction(h, x, h->w.corr))) return rc;
  if (prec == KFBI_FP64) {
    SolveArgs sa;
    sa.src = f_dev;
    sa.corr = h->w.corr;
    sa.lambda = lambda;
    sa.out_user = u_dev;
    if ((rc = box_solve64(h, sa, h->w.grid64))) return rc;
    // true residual g^N - du^+/dn relative to ||g||
    if ((rc = launch_limit64(h, h->w.grid64, x, gN_dev, -1.0, h->w.r))) return rc;
  } else {
    if ((rc = refined_solve(h, f_dev, 1.0, h->w.corr, lambda, u_dev))) return rc;
    if ((rc = launch_limit_user(h, u_dev, x, gN_dev, -1.0, h->w.r))) return rc;
  }
  double rn, gn;
  double* slot = h->w.small + small_nrm2(h->opts.restart);
  if ((rc = norm2(h, h->w.r, slot, &rn))) return rc;
  if ((rc = norm2(h, h->w.g, slot, &gn))) return rc;
  st.true_rel_res = gn > 0 ? rn / gn : rn;
  {
    int herr = 0;
    KFBI_CUDA(cudaMemcpyAsync(&herr, h->w.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    KFBI_CUDA(cudaStreamSynchronize(h->stream));
    if (herr & DEVERR_TIMEOUT) {
      set_error("a bounded wait on a TMA transfer gave up; results are invalid");
      return KFBI_ERR_CUDA;
    }
  }
  st.ms = elapsed_ms(t0);
  if (stats) *stats = st;
  return solve_rc;
}

// The Strang steps of bidomain_step; istim (may be NULL) is the extracellular
// stimulus: it adds beta I / sigma_e to the V problem's source, and the
// Poisson problem Lap S = -beta I (solved once per call, the stimulus does
// not change with time) gives the extracellular potential.
static int bidomain_impl(kfbi_handle* h, const kfbi_fhn* p, const double* istim, double* V_dev, double* w_dev,
                         double* ue_dev, int nsteps, kfbi_stats* per_step) {
  if (int rc = check_handle(h)) return rc;
  if (!p || !V_dev || !w_dev || nsteps < 0) {
    set_error("null argument");
    return KFBI_ERR_ARG;
  }
  const int64_t n = grid_points(h);
  const double lam = (2.0 * p->Cm * p->beta / h->dt) * (1.0 / h->sigma_i + 1.0 / h->sigma_e);
  const double k = 0.5 * h->dt;
  int rc;
  int final_rc = KFBI_OK;
  if (istim != nullptr) {
    const int M = h->t.M;
    if (!h->w.fsrc && (rc = dalloc(h, &h->w.fsrc, (size_t)n))) return rc;
    if (!h->w.S64 && (rc = dalloc(h, &h->w.S64, (size_t)n))) return rc;
    if (!h->w.psiS && (rc = dalloc(h, &h->w.psiS, (size_t)M))) return rc;
    if (!h->w.zeroM && (rc = dalloc(h, &h->w.zeroM, (size_t)M))) return rc;
    KFBI_CUDA(cudaMemsetAsync(h->w.zeroM, 0, sizeof(double) * (size_t)M, h->stream));
    KFBI_CUDA(cudaMemsetAsync(h->w.psiS, 0, sizeof(double) * (size_t)M, h->stream));
    // S problem: Lap S = -beta I, homogeneous Neumann data, lambda = 0
    if ((rc = launch_stim_source(h, nullptr, 0.0, istim, -p->beta, h->w.fsrc, n))) return rc;
    kfbi_stats sst{};
    rc = kfbi_solve_neumann(h, 0.0, h->w.fsrc, h->w.zeroM, h->w.S64, h->w.psiS, &sst);
    if (rc != KFBI_OK && rc != KFBI_ERR_NOT_CONVERGED) return rc;
    if (rc == KFBI_ERR_NOT_CONVERGED) final_rc = rc;
  }
  KFBI_CUDA(cudaMemsetAsync(h->w.err, 0, sizeof(int), h->stream));
  // per step: ||g^N - du^+/dn||^2 and ||g||^2 (true residual, read once at
  // the end) and, with per_step, CUDA events between the phases
  if (nsteps > h->step_cap) {
    if (h->w.step_sq) cudaFree(h->w.step_sq);
    h->w.step_sq = nullptr;
    h->step_cap = 0;
    KFBI_CUDA(cudaMalloc((void**)&h->w.step_sq, sizeof(double) * 2 * (size_t)nsteps));
    h->step_cap = nsteps;
  }
  constexpr int NEV = 7;
  const bool timed = per_step != nullptr;
  while (timed && h->step_events.size() < (size_t)NEV * nsteps) {
    cudaEvent_t e;
    KFBI_CUDA(cudaEventCreate(&e));
    h->step_events.push_back(e);
  }
  std::vector<kfbi_stats> stats((size_t)nsteps);
  auto mark = [&](int s, int k) -> int {
    if (timed) KFBI_CUDA(cudaEventRecord(h->step_events[(size_t)NEV * s + k], h->stream));
    return KFBI_OK;
  };
  for (int s = 0; s < nsteps; ++s) {
    kfbi_stats& st = stats[s];
    auto t0 = std::chrono::steady_clock::now();
    if ((rc = mark(s, 0))) return rc;
    // the forward half step of steps after the first ran in the previous
    // step's backward pass
    if (s == 0 && (rc = launch_react_fe(p, k, V_dev, w_dev, n, h->stream))) return rc;
    if ((rc = mark(s, 1))) return rc;
    const int prec = h->opts.precision == KFBI_FP64 ? KFBI_FP64 : KFBI_MIXED;
    // source of the V problem: -lam V (+ beta I / sigma_e with a stimulus)
    const double* vsrc = V_dev;
    double alpha = -lam;
    if (istim != nullptr) {
      if ((rc = launch_stim_source(h, V_dev, lam, istim, p->beta / h->sigma_e, h->w.fsrc, n))) return rc;
      vsrc = h->w.fsrc;
      alpha = 1.0;
    }
    // g = -dv_V^+/dn with v_V = L_h^{-1}(source)
    rc = prec == KFBI_FP64 ? rhs_g(h, lam, vsrc, alpha, nullptr, h->w.g)
                           : rhs_g_acc(h, lam, vsrc, alpha, nullptr, h->w.g);
    if (rc) return rc;
    if ((rc = mark(s, 2))) return rc;
    // initial density: the previous one, or the learned prediction when its
    // float32 residual is smaller
    if ((rc = vec_copy(h, h->w.psi_save, h->w.psi_prev, h->t.M))) return rc;
    const double* fallback = nullptr;
    const double* fallback_res2 = nullptr;
    double gnorm = -1.0;
    const bool learned = h->opts.precision == KFBI_MIXED_LEARNED && h->warm != nullptr;
    h->proj_valid = false;
    if ((h->opts.warm == KFBI_WARM_PROJECTION || learned) && h->opts.solver == KFBI_GMRES && h->hist_count >= 1) {
      h->proj_valid = true;
      // psi_F from the history, then one step of the simple iteration
      // psi_F + 2 gamma r_F; psi_F itself (residual known) is the fallback
      const int M = h->t.M;
      if ((rc = project_history(h, h->w.g, &gnorm, &fallback_res2))) return rc;
      if (learned && h->grid.dim == 3) {
        // the network corrects psi_F + 2 gamma r_F in units of rms(r_F)
        // (||r_F||^2 and ||g||^2 are already in sq[1], sq[2])
        double* sq = h->w.proj + KFBI_HISTORY * (KFBI_HISTORY + 2);
        if ((rc = vec_dots(h, h->w.psiF, 1, M, h->w.psiF, sq))) return rc;
        if ((rc = mlp_warmstart(h->warm, h->stream, h->w.psiF, h->w.rF, h->w.g, sq, h->t.nodes, h->t.n_normal, M,
                                2.0 * h->opts.gamma, h->w.psi_prev)))
          return rc;
        st.warmstart = 1;
      } else {
        if ((rc = vec_copy(h, h->w.psi_prev, h->w.psiF, M))) return rc;
        if ((rc = vec_axpby(h, h->w.psi_prev, 2.0 * h->opts.gamma, h->w.rF, 1.0, M))) return rc;
      }
      fallback = h->w.psiF;
    }
    // the guess as it enters the solver (kfbi_get_warm_guess)
    if ((rc = vec_copy(h, h->w.psi_learn, h->w.psi_prev, h->t.M))) return rc;
    if ((rc = mark(s, 3))) return rc;
    // mixed forms: the history holds exact images A psi_s, so r_F is the
    // float64-accurate residual of psi_F
    const bool ir = prec != KFBI_FP64 && h->opts.solver == KFBI_GMRES;
    const int src = solve_bie(h, prec, lam, h->w.g, h->w.psi_prev, &st, fallback, fallback_res2, gnorm,
                              ir ? h->w.rF : nullptr);
    if (src != KFBI_OK && src != KFBI_ERR_NOT_CONVERGED) return src;
    if ((rc = vec_copy(h, h->w.psi_prev2, h->w.psi_save, h->t.M))) return rc;
    if ((rc = vec_copy(h, h->w.g_prev, h->w.g, h->t.M))) return rc;
    if ((rc = push_history(h, h->w.psi_prev, h->w.g, ir ? h->w.r2 : nullptr))) return rc;
    ++h->n_hist;
    if (src == KFBI_ERR_NOT_CONVERGED) final_rc = src;
    if ((rc = mark(s, 4))) return rc;
    // V <- 2 (v_V + v_B(psi)) - V, and the true residual g^N - du^+/dn of
    // u = v_V + v_B(psi) at the nodes (homogeneous Neumann data: g^N = 0)
    const double* x;
    if ((rc = density_vector(h, h->w.psi_prev, &x))) return rc;
    if (prec == KFBI_FP64) {
      // one float64 solve of the combined right-hand side; the padded work
      // grid keeps u for the limit
      if ((rc = launch_correction(h, x, h->w.corr))) return rc;
      SolveArgs sa;
      sa.src = vsrc;
      sa.alpha = alpha;
      sa.corr = h->w.corr;
      sa.lambda = lam;
      sa.out_user = V_dev;
      sa.aux = V_dev;
      sa.beta = 2.0;
      sa.gamma = -1.0;
      if ((rc = box_solve64(h, sa, h->w.grid64))) return rc;
      if ((rc = launch_limit64(h, h->w.grid64, x, nullptr, -1.0, h->w.tmp))) return rc;
    } else {
      // the refined solver's last act was the float64-accurate residual at
      // the final density, which left v_B(psi) in u64; v_V is in vV64.  The
      // midpoint 2 (v_V + v_B) - V is formed by the backward-Euler pass below
      // (nothing reads V in between)
      if ((rc = launch_limit_user(h, h->w.vV64, nullptr, nullptr, -1.0, h->w.tmp))) return rc;
      if ((rc = launch_limit_user(h, h->w.u64, x, h->w.tmp, -1.0, h->w.tmp))) return rc;
    }
    if ((rc = vec_dots(h, h->w.tmp, 1, h->t.M, h->w.tmp, h->w.step_sq + 2 * s))) return rc;
    if ((rc = vec_dots(h, h->w.g, 1, h->t.M, h->w.g, h->w.step_sq + 2 * s + 1))) return rc;
    if ((rc = mark(s, 5))) return rc;
    // backward half step, and the next step's forward half step in the same
    // pass (not after the last step)
    const bool fe_next = s + 1 < nsteps;
    if (prec == KFBI_FP64) {
      if ((rc = launch_react_be(p, k, V_dev, w_dev, n, h->w.err, h->stream, nullptr, nullptr, fe_next))) return rc;
    } else if ((rc = launch_react_be(p, k, V_dev, w_dev, n, h->w.err, h->stream, h->w.vV64, h->w.u64, fe_next))) {
      return rc;
    }
    if ((rc = mark(s, 6))) return rc;
    st.ms = elapsed_ms(t0);
  }
  if (ue_dev) {
    if ((rc = istim != nullptr ? launch_ue_S(h, V_dev, h->w.S64, ue_dev) : launch_ue(h, V_dev, ue_dev))) return rc;
  }
  int herr = 0;
  std::vector<double> sq((size_t)2 * nsteps + 1);
  KFBI_CUDA(cudaMemcpyAsync(&herr, h->w.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  if (nsteps > 0)
    KFBI_CUDA(cudaMemcpyAsync(sq.data(), h->w.step_sq, sizeof(double) * 2 * (size_t)nsteps, cudaMemcpyDeviceToHost,
                              h->stream));
  KFBI_CUDA(cudaStreamSynchronize(h->stream));
  for (int s = 0; s < nsteps; ++s) {
    kfbi_stats& st = stats[s];
    const double rr = std::sqrt(sq[2 * s]), gg = std::sqrt(sq[2 * s + 1]);
    st.true_rel_res = gg > 0.0 ? rr / gg : rr;
    if (timed) {
      float t[NEV - 1];
      for (int q = 0; q + 1 < NEV; ++q)
        KFBI_CUDA(cudaEventElapsedTime(&t[q], h->step_events[(size_t)NEV * s + q], h->step_events[(size_t)NEV * s + q + 1]));
      st.react_ms = t[0] + t[5];
      st.rhs_ms = t[1];
      st.warm_ms = t[2];
      st.solve_ms = t[3];
      st.assemble_ms = t[4];
      per_step[s] = st;
    }
  }
  if (herr & DEVERR_TIMEOUT) {
    set_error("a bounded wait on a TMA transfer gave up; results are invalid");
    return KFBI_ERR_CUDA;
  }
  if (herr & DEVERR_NEWTON) {
    set_error("backward-Euler Newton iteration hit its cap");
    return KFBI_ERR_NEWTON;
  }
  return final_rc;
}

// Strang steps with the coupled anisotropic diffusion step: forward-Euler
// reaction over dt/2; the backward-Euler half step of Eq. pde1 with kappa =
// Cm beta / (dt/2), f = (-kappa V, kappa V - beta I), solved for (Phi_i,
// Phi_e) by GMRES on the density pair (warm start: the previous pair); V <-
// 2 (Phi_i - Phi_e) - V; backward-Euler reaction over dt/2.  ue_dev receives
// the last solve's Phi_e (the midpoint level) with zero mean over Omega.
static int bidomain_coupled_impl(kfbi_handle* h, const kfbi_fhn* p, const double* istim, double* V_dev,
                                 double* w_dev, double* ue_dev, int nsteps, kfbi_stats* per_step) {
  if ((h->opts.precision != KFBI_FP64 && h->opts.precision != KFBI_MIXED) || h->opts.solver != KFBI_GMRES) {
    set_error("the coupled system is solved with GMRES, in float64 or with float32 transforms");
    return KFBI_ERR_ARG;
  }
  const int prec = h->opts.precision;
  const int64_t n = grid_points(h);
  const int M = h->t.M, nk = h->nk;
  const double kap = p->Cm * p->beta / (0.5 * h->dt);
  const double k = 0.5 * h->dt;
  int rc, final_rc = KFBI_OK;
  if (istim != nullptr && !h->w.fsrc && (rc = dalloc(h, &h->w.fsrc, (size_t)n))) return rc;
  if (!h->w.zeroM) {
    if ((rc = dalloc(h, &h->w.zeroM, (size_t)M))) return rc;
    KFBI_CUDA(cudaMemsetAsync(h->w.zeroM, 0, sizeof(double) * (size_t)M, h->stream));
  }
  KFBI_CUDA(cudaMemsetAsync(h->w.err, 0, sizeof(int), h->stream));
  if (nsteps > h->step_cap) {
    if (h->w.step_sq) cudaFree(h->w.step_sq);
    h->w.step_sq = nullptr;
    h->step_cap = 0;
    KFBI_CUDA(cudaMalloc((void**)&h->w.step_sq, sizeof(double) * 2 * (size_t)nsteps));
    h->step_cap = nsteps;
  }
  constexpr int NEV = 7;
  const bool timed = per_step != nullptr;
  while (timed && h->step_events.size() < (size_t)NEV * nsteps) {
    cudaEvent_t e;
    KFBI_CUDA(cudaEventCreate(&e));
    h->step_events.push_back(e);
  }
  auto mark = [&](int s, int q) -> int {
    if (timed) KFBI_CUDA(cudaEventRecord(h->step_events[(size_t)NEV * s + q], h->stream));
    return KFBI_OK;
  };
  std::vector<kfbi_stats> stats((size_t)nsteps);
  double* phi_i = h->w.u64;
  double* phi_e = h->w.vV64;
  for (int s = 0; s < nsteps; ++s) {
    kfbi_stats& st = stats[s];
    auto t0 = std::chrono::steady_clock::now();
    if ((rc = mark(s, 0))) return rc;
    // after the first step the forward half step ran in the previous
    // step's backward pass
    if (s == 0 && (rc = launch_react_fe(p, k, V_dev, w_dev, n, h->stream))) return rc;
    if ((rc = mark(s, 1))) return rc;
    // f_i = -kappa V, f_e = kappa V (- beta I)
    const double* src_e = V_dev;
    double a_e = kap;
    if (istim != nullptr) {
      if ((rc = launch_stim_source(h, V_dev, -kap, istim, -p->beta, h->w.fsrc, n))) return rc;
      src_e = h->w.fsrc;
      a_e = 1.0;
    }
    rc = prec == KFBI_FP64 ? rhs_g_coupled(h, kap, V_dev, -kap, src_e, a_e, h->w.zeroM, h->w.zeroM, h->w.g)
                           : rhs_g_acc_coupled(h, kap, V_dev, -kap, src_e, a_e, h->w.zeroM, h->w.zeroM, h->w.g);
    if (rc) return rc;
    if ((rc = mark(s, 2))) return rc;
    if ((rc = vec_copy(h, h->w.psi_save, h->w.psi_prev, nk))) return rc;
    // initial density pair: the previous one, or (KFBI_WARM_PROJECTION) the
    // history projection plus one step of the simple iteration, with the
    // projection itself as the fallback the first residual decides on
    const double* fallback = nullptr;
    const double* fallback_res2 = nullptr;
    double gnorm = -1.0;
    h->proj_valid = false;
    if (h->opts.warm == KFBI_WARM_PROJECTION && h->hist_count >= 1) {
      h->proj_valid = true;
      if ((rc = project_history(h, h->w.g, &gnorm, &fallback_res2))) return rc;
      if ((rc = vec_copy(h, h->w.psi_prev, h->w.psiF, nk))) return rc;
      if ((rc = vec_axpby(h, h->w.psi_prev, 2.0 * h->opts.gamma, h->w.rF, 1.0, nk))) return rc;
      fallback = h->w.psiF;
    }
    if ((rc = vec_copy(h, h->w.psi_learn, h->w.psi_prev, nk))) return rc;
    if ((rc = mark(s, 3))) return rc;
    const bool ir = prec != KFBI_FP64;
    const int src = solve_bie(h, prec, kap, h->w.g, h->w.psi_prev, &st, fallback, fallback_res2, gnorm,
                              ir ? h->w.rF : nullptr);
    if (src != KFBI_OK && src != KFBI_ERR_NOT_CONVERGED) return src;
    if (src == KFBI_ERR_NOT_CONVERGED) final_rc = src;
    if ((rc = vec_copy(h, h->w.psi_prev2, h->w.psi_save, nk))) return rc;
    if ((rc = vec_copy(h, h->w.g_prev, h->w.g, nk))) return rc;
    if ((rc = push_history(h, h->w.psi_prev, h->w.g, ir ? h->w.r2 : nullptr))) return rc;
    ++h->n_hist;
    if ((rc = mark(s, 4))) return rc;
    if (prec == KFBI_FP64) {
      if ((rc = assemble_coupled(h, kap, V_dev, -kap, src_e, a_e, h->w.psi_prev, h->w.zeroM, h->w.zeroM, phi_i,
                                 phi_e, h->w.tmp)))
        return rc;
      if ((rc = launch_midpoint_diff(h, V_dev, phi_i, phi_e, n))) return rc;
    } else {
      // GMRES-IR's last act was the refined residual at the final density:
      // v_B of both components in u64, u64b, v_V in vV64, vV64b
      if ((rc = launch_midpoint4(h, V_dev, h->w.vV64, h->w.u64, h->w.vV64b, h->w.u64b, n))) return rc;
      if ((rc = true_residual_coupled_acc(h, h->w.psi_prev, h->w.zeroM, h->w.zeroM, h->w.tmp))) return rc;
    }
    if ((rc = vec_dots(h, h->w.tmp, 1, nk, h->w.tmp, h->w.step_sq + 2 * s))) return rc;
    if ((rc = vec_dots(h, h->w.g, 1, nk, h->w.g, h->w.step_sq + 2 * s + 1))) return rc;
    if ((rc = mark(s, 5))) return rc;
    if ((rc = launch_react_be(p, k, V_dev, w_dev, n, h->w.err, h->stream, nullptr, nullptr, s + 1 < nsteps)))
      return rc;
    if ((rc = mark(s, 6))) return rc;
    st.ms = elapsed_ms(t0);
  }
  if (ue_dev && prec != KFBI_FP64 && nsteps > 0) {
    // Phi_e = v_V + v_B of the extracellular component (the last solve)
    KFBI_CUDA(cudaMemcpyAsync(ue_dev, h->w.vV64b, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, h->stream));
    if ((rc = launch_lincomb(h, ue_dev, 1.0, h->w.u64b, 1.0, n))) return rc;
    if ((rc = launch_sub_mean(h, ue_dev, ue_dev))) return rc;
  } else if (ue_dev && (rc = launch_sub_mean(h, phi_e, ue_dev))) {
    return rc;
  }
  int herr = 0;
  std::vector<double> sq((size_t)2 * nsteps + 1);
  KFBI_CUDA(cudaMemcpyAsync(&herr, h->w.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  if (nsteps > 0)
    KFBI_CUDA(cudaMemcpyAsync(sq.data(), h->w.step_sq, sizeof(double) * 2 * (size_t)nsteps, cudaMemcpyDeviceToHost,
                              h->stream));
  KFBI_CUDA(cudaStreamSynchronize(h->stream));
  for (int s = 0; s < nsteps; ++s) {
    kfbi_stats& st = stats[s];
    const double rr = std::sqrt(sq[2 * s]), gg = std::sqrt(sq[2 * s + 1]);
    st.true_rel_res = gg > 0.0 ? rr / gg : rr;
    if (timed) {
      float t[NEV - 1];
      for (int q = 0; q + 1 < NEV; ++q)
        KFBI_CUDA(cudaEventElapsedTime(&t[q], h->step_events[(size_t)NEV * s + q], h->step_events[(size_t)NEV * s + q + 1]));
      st.react_ms = t[0] + t[5];
      st.rhs_ms = t[1];
      st.warm_ms = t[2];
      st.solve_ms = t[3];
      st.assemble_ms = t[4];
      per_step[s] = st;
    }
  }
  if (herr & DEVERR_NEWTON) {
    set_error("backward-Euler Newton iteration hit its cap");
    return KFBI_ERR_NEWTON;
  }
  return final_rc;
}

int bidomain_step(kfbi_handle* h, const kfbi_fhn* p, double* V_dev, double* w_dev, double* ue_dev, int nsteps,
                  kfbi_stats* per_step) {
  if (h != nullptr && h->coupled) {
    if (!p || !V_dev || !w_dev || nsteps < 0) {
      set_error("null argument");
      return KFBI_ERR_ARG;
    }
    return bidomain_coupled_impl(h, p, nullptr, V_dev, w_dev, ue_dev, nsteps, per_step);
  }
  return bidomain_impl(h, p, nullptr, V_dev, w_dev, ue_dev, nsteps, per_step);
}

int kfbi_solve_coupled(kfbi_handle* h, double kappa, const double* fi_dev, const double* fe_dev,
                       const double* gNi_dev, const double* gNe_dev, double* phi_i_dev, double* phi_e_dev,
                       double* psi_dev, kfbi_stats* stats) {
  if (int rc = check_handle(h)) return rc;
  if (!h->coupled || !fi_dev || !fe_dev || !gNi_dev || !gNe_dev || !phi_i_dev || !phi_e_dev || !psi_dev ||
      !(kappa > 0.0)) {
    set_error("kfbi_solve_coupled needs a coupled handle, kappa > 0 and every field");
    return KFBI_ERR_ARG;
  }
  kfbi_stats st{};
  auto t0 = std::chrono::steady_clock::now();
  int rc;
  const int prec = h->opts.precision == KFBI_FP64 ? KFBI_FP64 : KFBI_MIXED;
  rc = prec == KFBI_FP64 ? rhs_g_coupled(h, kappa, fi_dev, 1.0, fe_dev, 1.0, gNi_dev, gNe_dev, h->w.g)
                         : rhs_g_acc_coupled(h, kappa, fi_dev, 1.0, fe_dev, 1.0, gNi_dev, gNe_dev, h->w.g);
  if (rc) return rc;
  const int solve_rc = solve_bie(h, prec, kappa, h->w.g, psi_dev, &st);
  if (solve_rc != KFBI_OK && solve_rc != KFBI_ERR_NOT_CONVERGED) return solve_rc;
  if (prec == KFBI_FP64) {
    if ((rc = assemble_coupled(h, kappa, fi_dev, 1.0, fe_dev, 1.0, psi_dev, gNi_dev, gNe_dev, phi_i_dev, phi_e_dev,
                               h->w.r)))
      return rc;
  } else {
    // (Phi_i, Phi_e) = v_V + v_B from the refined solves GMRES-IR left
    const int64_t n = grid_points(h);
    KFBI_CUDA(cudaMemcpyAsync(phi_i_dev, h->w.vV64, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, h->stream));
    KFBI_CUDA(cudaMemcpyAsync(phi_e_dev, h->w.vV64b, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, h->stream));
    if ((rc = launch_lincomb(h, phi_i_dev, 1.0, h->w.u64, 1.0, n))) return rc;
    if ((rc = launch_lincomb(h, phi_e_dev, 1.0, h->w.u64b, 1.0, n))) return rc;
    if ((rc = true_residual_coupled_acc(h, psi_dev, gNi_dev, gNe_dev, h->w.r))) return rc;
  }
  double rn, gn;
  double* slot = h->w.small + small_nrm2(h->opts.restart);
  if ((rc = norm2(h, h->w.r, slot, &rn))) return rc;
  if ((rc = norm2(h, h->w.g, slot, &gn))) return rc;
  st.true_rel_res = gn > 0 ? rn / gn : rn;
  st.ms = elapsed_ms(t0);
  if (stats) *stats = st;
  return solve_rc;
}

int kfbi_box_solve_coupled(kfbi_handle* h, double kappa, const double* ri_dev, const double* re_dev, double* vi_dev,
                           double* ve_dev) {
  if (int rc = check_handle(h)) return rc;
  if (!h->coupled || !ri_dev || !re_dev || !vi_dev || !ve_dev) {
    set_error("kfbi_box_solve_coupled needs a coupled handle and every field");
    return KFBI_ERR_ARG;
  }
  SolveArgs si, se;
  si.src = ri_dev;
  si.out_user = vi_dev;
  se.src = re_dev;
  se.out_user = ve_dev;
  Coupling cp = h->cpl;
  cp.kappa = kappa;
  return box_solve_coupled64(h, si, se, cp, h->w.grid64, h->w.grid64b);
}

int kfbi_apply_A_coupled(kfbi_handle* h, double kappa, const double* psi_dev, double* out_dev) {
  if (int rc = check_handle(h)) return rc;
  if (!h->coupled || !psi_dev || !out_dev) {
    set_error("kfbi_apply_A_coupled needs a coupled handle");
    return KFBI_ERR_ARG;
  }
  return apply_A_coupled(h, kappa, psi_dev, out_dev, 1.0, nullptr);
}

int kfbi_bidomain_step_stim(kfbi_handle* h, const kfbi_fhn* p, const double* istim_dev, double* V_dev,
                            double* w_dev, double* ue_dev, int nsteps, kfbi_stats* per_step) {
  if (h != nullptr && neumann_box(h) && istim_dev != nullptr) {
    set_error("the stimulus's Poisson problem has no Neumann-box Green's function (lambda = 0)");
    return KFBI_ERR_ARG;
  }
  if (h != nullptr && h->coupled) {
    if (!p || !V_dev || !w_dev || nsteps < 0) {
      set_error("null argument");
      return KFBI_ERR_ARG;
    }
    return bidomain_coupled_impl(h, p, istim_dev, V_dev, w_dev, ue_dev, nsteps, per_step);
  }
  return bidomain_impl(h, p, istim_dev, V_dev, w_dev, ue_dev, nsteps, per_step);
}

int kfbi_set_warmstart(kfbi_handle* h, kfbi_mlp* m) {
  if (int rc = check_handle(h)) return rc;
  if (m != nullptr && h->grid.dim != 3) {
    set_error("the learned warm start needs a 3-D geometry");
    return KFBI_ERR_ARG;
  }
  h->warm = m;
  return KFBI_OK;
}

int kfbi_get_densities(kfbi_handle* h, double* psi_dev, double* psi_prev_dev, double* g_dev) {
  if (int rc = check_handle(h)) return rc;
  const size_t n = sizeof(double) * (size_t)h->nk;
  if (psi_dev) KFBI_CUDA(cudaMemcpyAsync(psi_dev, h->w.psi_prev, n, cudaMemcpyDeviceToDevice, h->stream));
  if (psi_prev_dev) KFBI_CUDA(cudaMemcpyAsync(psi_prev_dev, h->w.psi_prev2, n, cudaMemcpyDeviceToDevice, h->stream));
  if (g_dev) KFBI_CUDA(cudaMemcpyAsync(g_dev, h->w.g, n, cudaMemcpyDeviceToDevice, h->stream));
  return KFBI_OK;
}

int kfbi_set_densities(kfbi_handle* h, const double* psi_dev, const double* psi_prev_dev, const double* g_dev,
                       int n_solves) {
  if (int rc = check_handle(h)) return rc;
  if (n_solves < 0) {
    set_error("negative solve count");
    return KFBI_ERR_ARG;
  }
  const size_t n = sizeof(double) * (size_t)h->nk;
  if (n_solves == 0) {
    KFBI_CUDA(cudaMemsetAsync(h->w.psi_prev, 0, n, h->stream));
    KFBI_CUDA(cudaMemsetAsync(h->w.psi_prev2, 0, n, h->stream));
    KFBI_CUDA(cudaMemsetAsync(h->w.g_prev, 0, n, h->stream));
  } else {
    if (!psi_dev || !psi_prev_dev || !g_dev) {
      set_error("null density history");
      return KFBI_ERR_ARG;
    }
    KFBI_CUDA(cudaMemcpyAsync(h->w.psi_prev, psi_dev, n, cudaMemcpyDeviceToDevice, h->stream));
    KFBI_CUDA(cudaMemcpyAsync(h->w.psi_prev2, psi_prev_dev, n, cudaMemcpyDeviceToDevice, h->stream));
    KFBI_CUDA(cudaMemcpyAsync(h->w.g_prev, g_dev, n, cudaMemcpyDeviceToDevice, h->stream));
    KFBI_CUDA(cudaMemcpyAsync(h->w.g, g_dev, n, cudaMemcpyDeviceToDevice, h->stream));
  }
  h->n_hist = n_solves;
  h->hist_count = 0;  // the projection history starts again from this state
  return KFBI_OK;
}

int kfbi_get_history(kfbi_handle* h, double* psi_hist_dev, double* g_hist_dev, int* n_solves) {
  if (int rc = check_handle(h)) return rc;
  const size_t n = sizeof(double) * (size_t)KFBI_HISTORY * h->nk;
  if (psi_hist_dev) KFBI_CUDA(cudaMemcpyAsync(psi_hist_dev, h->w.hist_psi, n, cudaMemcpyDeviceToDevice, h->stream));
  if (g_hist_dev) KFBI_CUDA(cudaMemcpyAsync(g_hist_dev, h->w.hist_g, n, cudaMemcpyDeviceToDevice, h->stream));
  if (n_solves) *n_solves = h->hist_count;
  return KFBI_OK;
}

int kfbi_set_history(kfbi_handle* h, const double* psi_hist_dev, const double* g_hist_dev, int n_solves) {
  if (int rc = check_handle(h)) return rc;
  if (n_solves < 0 || (n_solves > 0 && (!psi_hist_dev || !g_hist_dev))) {
    set_error("bad density history");
    return KFBI_ERR_ARG;
  }
  const int M = h->nk;
  const size_t n = sizeof(double) * (size_t)KFBI_HISTORY * M;
  if (n_solves > 0) {
    KFBI_CUDA(cudaMemcpyAsync(h->w.hist_psi, psi_hist_dev, n, cudaMemcpyDeviceToDevice, h->stream));
    KFBI_CUDA(cudaMemcpyAsync(h->w.hist_g, g_hist_dev, n, cudaMemcpyDeviceToDevice, h->stream));
    // the previous-density state follows from the two latest slots
    const size_t s1 = (size_t)((n_solves - 1) % KFBI_HISTORY) * M;
    int rc;
    if ((rc = vec_copy(h, h->w.psi_prev, h->w.hist_psi + s1, M))) return rc;
    if ((rc = vec_copy(h, h->w.g, h->w.hist_g + s1, M))) return rc;
    if ((rc = vec_copy(h, h->w.g_prev, h->w.hist_g + s1, M))) return rc;
    if (n_solves >= 2) {
      const size_t s2 = (size_t)((n_solves - 2) % KFBI_HISTORY) * M;
      if ((rc = vec_copy(h, h->w.psi_prev2, h->w.hist_psi + s2, M))) return rc;
    } else {
      KFBI_CUDA(cudaMemsetAsync(h->w.psi_prev2, 0, sizeof(double) * (size_t)M, h->stream));
    }
  } else {
    KFBI_CUDA(cudaMemsetAsync(h->w.psi_prev, 0, sizeof(double) * (size_t)M, h->stream));
    KFBI_CUDA(cudaMemsetAsync(h->w.psi_prev2, 0, sizeof(double) * (size_t)M, h->stream));
    KFBI_CUDA(cudaMemsetAsync(h->w.g_prev, 0, sizeof(double) * (size_t)M, h->stream));
  }
  h->hist_count = n_solves;
  h->n_hist = n_solves;
  return KFBI_OK;
}

int kfbi_get_projection(kfbi_handle* h, double* psiF_dev, double* rF_dev) {
  if (int rc = check_handle(h)) return rc;
  const size_t n = sizeof(double) * (size_t)h->nk;
  if (psiF_dev) KFBI_CUDA(cudaMemcpyAsync(psiF_dev, h->w.psiF, n, cudaMemcpyDeviceToDevice, h->stream));
  if (rF_dev) KFBI_CUDA(cudaMemcpyAsync(rF_dev, h->w.rF, n, cudaMemcpyDeviceToDevice, h->stream));
  return KFBI_OK;
}

int kfbi_get_warm_guess(kfbi_handle* h, double* psi0_dev) {
  if (int rc = check_handle(h)) return rc;
  if (!psi0_dev) {
    set_error("null output");
    return KFBI_ERR_ARG;
  }
  KFBI_CUDA(cudaMemcpyAsync(psi0_dev, h->w.psi_learn, sizeof(double) * (size_t)h->nk, cudaMemcpyDeviceToDevice,
                            h->stream));
  return KFBI_OK;
}

int kfbi_training_rows(kfbi_handle* h, float* F_dev, float* T_dev) {
  if (int rc = check_handle(h)) return rc;
  if (!F_dev || !T_dev || h->grid.dim != 3) {
    set_error("null output, or a 2-D handle (the network reads 3-D nodes and normals)");
    return KFBI_ERR_ARG;
  }
  if (!h->proj_valid) {
    set_error("the last Strang step did not start from the history projection");
    return KFBI_ERR_ARG;
  }
  const int M = h->t.M;
  // the sums of squares of the projection step: ||r_F||^2 and ||g||^2 from
  // the projection, ||psi_F||^2 as the learned form computes it, so that the
  // rows equal the network's inference input of that step
  double* sq = h->w.proj + KFBI_HISTORY * (KFBI_HISTORY + 2);
  int rc;
  if ((rc = vec_dots(h, h->w.psiF, 1, M, h->w.psiF, sq))) return rc;
  return launch_train_rows(h->stream, h->w.psi_prev, h->w.psiF, h->w.rF, h->w.g, sq, h->t.nodes, h->t.n_normal, M,
                           2.0 * h->opts.gamma, F_dev, T_dev);
}

int kfbi_transform_pass(kfbi_handle* h, int precision, int pass, double lambda) {
  if (int rc = check_handle(h)) return rc;
  if (pass < 0 || pass > 5) {
    set_error("pass must be 0..5");
    return KFBI_ERR_ARG;
  }
  if (neumann_box(h)) {
    set_error("single transform passes are those of the Dirichlet box");
    return KFBI_ERR_ARG;
  }
  return transform_pass(h, precision, pass, lambda);
}

int64_t kfbi_launch_count(void) { return (int64_t)g_launches.load(); }

int kfbi_react_fe(const kfbi_fhn* p, double k, double* V_dev, double* w_dev, int64_t n, void* stream) {
  if (!p || !V_dev || !w_dev || n < 0) {
    set_error("null argument");
    return KFBI_ERR_ARG;
  }
  return launch_react_fe(p, k, V_dev, w_dev, n, (cudaStream_t)stream);
}

int kfbi_react_be(const kfbi_fhn* p, double k, double* V_dev, double* w_dev, int64_t n, void* stream) {
  if (!p || !V_dev || !w_dev || n < 0) {
    set_error("null argument");
    return KFBI_ERR_ARG;
  }
  int* err = nullptr;
  KFBI_CUDA(cudaMallocAsync((void**)&err, sizeof(int), (cudaStream_t)stream));
  KFBI_CUDA(cudaMemsetAsync(err, 0, sizeof(int), (cudaStream_t)stream));
  int rc = launch_react_be(p, k, V_dev, w_dev, n, err, (cudaStream_t)stream);
  int herr = 0;
  cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  cudaFreeAsync(err, (cudaStream_t)stream);
  KFBI_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (rc) return rc;
  if (herr & DEVERR_NEWTON) {
    set_error("backward-Euler Newton iteration hit its cap");
    return KFBI_ERR_NEWTON;
  }
  return KFBI_OK;
}

}  // extern "C"
