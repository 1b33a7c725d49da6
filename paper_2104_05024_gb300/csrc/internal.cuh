// Internal declarations shared by the CUDA translation units of the KFBI
// library: the handle, device tables, launch helpers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "kfbi.h"

namespace kfbi {

constexpr int PATCH_MAX = 16;   // points of one local surface fit
constexpr int MAX_RESTART = 64;
#define KFBI_ARN_BLOCKS 608  // 4 x 152 SMs: row blocks of the single-launch Krylov reductions

// error-word bits written by device code
constexpr int DEVERR_GEOMETRY = 1;
constexpr int DEVERR_NEWTON = 2;
constexpr int DEVERR_SINGULAR = 4;
constexpr int DEVERR_TIMEOUT = 8;   // a bounded wait on a TMA transfer gave up

void set_error(const char* fmt, ...);

// Programmatic dependent launch.  The hot kernels of a solve and of a
// Krylov iteration are launched with programmatic stream serialization: a
// kernel may start while the one before it in the stream is still
// finishing, load its constant tables (twiddles, sines, mu1: written once at
// setup), and then wait in pdl_wait() until that predecessor has completed
// and its writes are visible.  Everything else it touches (grids, vectors,
// sources, corrections, the skip flag, mode-factor tables) it reads or
// writes only after the wait.  pdl_launch_next() lets the next kernel launch:
// kernels whose blocks are all resident at once (persistent passes, the
// single-wave Krylov and gather kernels) call it right after their wait,
// multi-wave passes at the end of each block, so a waiting successor never
// takes an SM from blocks of its predecessor that have not started.  Without
// the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename K, typename... Args>
cudaError_t launch_pdl(K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// error status of a failed launch (reads and clears the launch error)
inline int launch_failed(const char* what) {
  set_error("launch of the %s failed: %s", what, cudaGetErrorString(cudaGetLastError()));
  return KFBI_ERR_CUDA;
}

// kernels launched by this library (instrumentation for benchmarks)
extern std::atomic<long long> g_launches;
#define KFBI_COUNT(n) (::kfbi::g_launches.fetch_add((n), std::memory_order_relaxed))

#define KFBI_CUDA(call)                                                           \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      ::kfbi::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                        __FILE__, __LINE__);                                      \
      return KFBI_ERR_CUDA;                                                       \
    }                                                                             \
  } while (0)

#define KFBI_CHECK_LAUNCH() KFBI_CHECK_LAUNCH_N(1)
// after a launcher that issued n kernels: count them and surface launch errors
#define KFBI_CHECK_LAUNCH_N(n)                                                    \
  do {                                                                            \
    KFBI_COUNT(n);                                                                \
    cudaError_t e_ = cudaGetLastError();                                          \
    if (e_ != cudaSuccess) {                                                      \
      ::kfbi::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                      \
      return KFBI_ERR_CUDA;                                                       \
    }                                                                             \
  } while (0)

// Geometry parameters copied to the device (plain values, passed by value).
struct GeomParams {
  int dim, kind, n_comp;
  double p[16];
  int comp_map[KFBI_MAX_COMP];
  double comp_axes[KFBI_MAX_COMP][3];
  int comp_tri_offset[KFBI_MAX_COMP];
  int comp_vert_offset[KFBI_MAX_COMP];
  int cube_n;
};

struct GridParams {
  int dim, N;
  double lo, h;
  int bc = KFBI_BOX_DIRICHLET;  // box condition: field layout (N-1)^dim or (N+1)^dim
};

// field (user) layout of a grid: nodes per axis and the node index k of
// array index 0 (interior nodes of the Dirichlet box, all nodes of the
// Neumann box)
__host__ __device__ inline int field_n(const GridParams& g) { return g.bc == KFBI_BOX_NEUMANN ? g.N + 1 : g.N - 1; }
__host__ __device__ inline int field_first(const GridParams& g) { return g.bc == KFBI_BOX_NEUMANN ? 0 : 1; }
// row length of the work grid: N (Dirichlet, padded), N + 1 (Neumann, the
// field layout itself)
__host__ __device__ inline int work_n(const GridParams& g) { return g.bc == KFBI_BOX_NEUMANN ? g.N + 1 : g.N; }
__host__ __device__ inline int64_t field_count(const GridParams& g) {
  const int64_t n = field_n(g);
  return g.dim == 3 ? n * n * n : n * n;
}

// Sparse tables of the hot path (all device pointers).
struct Tables {
  // irregular nodes, increasing user-layout flat index
  int n_irr = 0;
  int32_t* irr = nullptr;
  int32_t* irr_arm = nullptr;     // [n_irr][6] arm codes: crossing*2 + end (end 0 = lower node)
  int8_t* irr_narm = nullptr;     // [n_irr]
  int32_t* line_start = nullptr;  // [(N-1)^(dim-1) + 1] first irregular index of each x-line
  // each irregular node's correction as one row on the density vector: the
  // rows of its crossing arms' end weights, concatenated (CSR)
  int32_t* cr_ptr = nullptr;      // [n_irr + 1]
  int32_t* cr_pid = nullptr;      // [nnz] density-vector indices
  double* cr_w = nullptr;         // [nnz] weights
  // crossings, sorted by (axis, lower node)
  int n_int = 0;
  int32_t* c_axis = nullptr;
  int32_t* c_lo = nullptr;        // user-layout flat index of the lower node
  int8_t* c_comp = nullptr;
  double* c_z = nullptr;
  int32_t* c_tri = nullptr;       // mesh-only domains: the triangle each crossing lies on
  int32_t* c_cnt = nullptr;       // entries of the crossing's density row
  int32_t* c_pid = nullptr;       // [n_int][PATCH_MAX] indices into x = psi (3-D) or [psi; m] (2-D)
  double* c_wlo = nullptr;        // [n_int][PATCH_MAX] correction weights for the lower node
  double* c_whi = nullptr;        // [n_int][PATCH_MAX] correction weights for the upper node
  // interface nodes
  int M = 0;
  int P = 0;                      // stencil points (6 or 10)
  int32_t* n_base = nullptr;      // padded-layout index of the stencil centre
  int8_t* n_sign = nullptr;       // [M][dim]
  int32_t* n_center = nullptr;    // [M][dim] 1-based node indices
  double* n_wn = nullptr;         // [M][P] weights of dv/dn on the stencil values
  int32_t* n_dcnt = nullptr;      // [M] entries of the node's jump row
  int32_t* n_dpid = nullptr;      // [M][PATCH_MAX + 1]
  double* n_dw = nullptr;         // [M][PATCH_MAX + 1]
  // 2-D periodic spline: moments m = G psi
  double* spline_G = nullptr;     // [M][M]
  // transform tables
  double* mu = nullptr;           // [N] eigenvalues of the 1-D second difference (index 0 unused)
  double* tw64 = nullptr;         // [2N] complex e^{i pi j / N}
  float* mu32 = nullptr;
  float* tw32 = nullptr;
  uint8_t* inside = nullptr;      // [(N-1)^dim] interior nodes
  // the same mask and the irregular nodes' flat indices on the field layout
  // (aliases of inside and irr for the Dirichlet box)
  uint8_t* inside_user = nullptr;
  int32_t* irr_user = nullptr;
  int n_inside = 0;
  double* nodes = nullptr;        // [M][dim] interface nodes
  double* n_normal = nullptr;     // [M][3] outward normals at the nodes
  double* ds = nullptr;           // [M] boundary quadrature weights
  double area = 0.0;              // their sum |Gamma|
  // diagonal conductivity of the component whose correction and limit rows
  // these are (1, 1, 1 for the scalar problem)
  double cond[3] = {1.0, 1.0, 1.0};
};

// coupled anisotropic system (Eq. pde1): per-axis conductivities of the two
// components and the coupling kappa; scale is set by the solver
struct Coupling {
  double di[3] = {1.0, 1.0, 1.0}, de[3] = {1.0, 1.0, 1.0};
  double kappa = 0.0, scale = 1.0;
};

struct Workspace {
  double* grid64 = nullptr;       // padded N^dim work grid
  double* grid64b = nullptr;      // second padded grid (volume solution)
  float* grid32 = nullptr;        // padded N^dim float grid
  double* corr = nullptr;         // [n_irr] correction values
  float* corr32 = nullptr;
  double* xvec = nullptr;         // [2M] density vector (psi, spline moments)
  double* vecs = nullptr;         // GMRES basis [(restart+1)][M] + scratch
  double* small = nullptr;        // GMRES Hessenberg/Givens on device
  double* partial = nullptr;      // reduction partial sums
  double* g = nullptr;            // [M]
  double* r = nullptr;            // [M]
  double* tmp = nullptr;          // [M]
  double* tmp2 = nullptr;         // [M]
  double* psi_prev = nullptr;     // [M] density of the previous diffusion solve
  double* r2 = nullptr;           // [M] outer residual of GMRES-IR
  double* psi_prev2 = nullptr;    // [M] density of the solve before the previous one
  double* psi_save = nullptr;     // [M]
  double* psi_learn = nullptr;    // [M] learned initial guess
  double* g_prev = nullptr;       // [M] right-hand side of the previous diffusion solve
  double* u64 = nullptr;          // user-layout float64 grid (refined solutions)
  double* res64 = nullptr;        // user-layout float64 grid (refinement residuals)
  double* vV64 = nullptr;         // user-layout float64 volume solution v_V of the step
  double* fsrc = nullptr;         // user-layout float64 source of a stimulated step
  double* S64 = nullptr;          // user-layout float64 S = sigma_i Phi_i + sigma_e Phi_e
  double* psiS = nullptr;         // [M] density of the S problem
  double* zeroM = nullptr;        // [M] zeros (homogeneous Neumann data)
  float* res32 = nullptr;         // user-layout float32 grid (refinement residuals)
  double* hist_psi = nullptr;     // [KFBI_HISTORY][M] densities of past solves
  double* hist_g = nullptr;       // [KFBI_HISTORY][M] their right-hand sides
  double* psiF = nullptr;         // [M] projected density
  double* rF = nullptr;           // [M] its residual
  double* proj = nullptr;         // Gram matrix, right side, coefficients
  double* host_small = nullptr;   // pinned host scalars
  int* err = nullptr;             // device error word
  int* stop = nullptr;            // Krylov stop flag (set by the Arnoldi step)
  unsigned* counter = nullptr;    // ticket counter of the single-launch reductions
  double* step_sq = nullptr;      // per Strang step: squared true residual, ||g||^2
  // coupled anisotropic system: second correction array, second 2-D density
  // vector, and (ds, ds) / 2 for its rank-one term
  double* corr2 = nullptr;
  double* xvec2 = nullptr;
  double* ds2 = nullptr;
  // coupled float32 forms: the second float grid and the extracellular
  // counterparts of u64 / vV64 / res64
  float* grid32b = nullptr;
  float* res32b = nullptr;
  double* u64b = nullptr;
  double* vV64b = nullptr;
  double* res64b = nullptr;
  int restart_cap = 0;
};

}  // namespace kfbi

struct kfbi_handle {
  kfbi::GeomParams gp;
  kfbi::GridParams grid;
  kfbi::Tables t;
  kfbi::Workspace w;
  kfbi_opts opts;
  double sigma_i, sigma_e, dt, lambda;
  cudaStream_t stream;
  size_t device_bytes = 0;
  std::vector<void*> allocations;
  bool have_prev = false;
  int n_hist = 0;                 // completed diffusion solves (density history)
  int hist_count = 0;             // solves held in the projection history ring
  bool proj_valid = false;        // the last Strang step started from the projection
  // coupled anisotropic system (kfbi_create_coupled): the rows of the
  // extracellular component in t2 (t holds the intracellular ones), the
  // conductivities, and the Krylov vector length nk = 2M (M otherwise)
  bool coupled = false;
  int cr_nnz = 0;                 // entries of the CSR correction rows
  kfbi::Coupling cpl;
  kfbi::Tables t2;
  int nk = 0;
  kfbi_mlp* warm = nullptr;       // learned warm start (not owned)
  // TMA descriptors of the float32 padded grid: [N x 32] tiles along y and z
  CUtensorMap tmap_y32, tmap_z32;
  CUtensorMap tmap_y32b, tmap_z32b;  // the same for the second float grid
  bool tma_b = false;
  bool tma = false;
  int sms = 152;                  // the device's multiprocessor count (persistent grids)
  bool xy_fused = false;          // float32 3-D solves use the cluster-fused x-y passes
  // float64 solves: the mode factors scale / mu_p for the lambda they were
  // built for (rinv_ok: the handle may allocate the table; set at creation)
  double* rinv64 = nullptr;
  double rinv_lambda = 0.0;
  bool rinv_ok = false;
  // coupled solves: the per-mode 2 x 2 solve factors for the kappa they were
  // built for, one table per element type (3 N^dim values each)
  double* cpl64 = nullptr;
  float* cpl32 = nullptr;
  double cpl64_kappa = 0.0, cpl32_kappa = 0.0;
  // device flag handed to the launches of a Krylov iteration enqueued ahead
  // of the host's convergence test (nullptr otherwise)
  const int* skip = nullptr;
  cudaEvent_t arn_ev[2] = {nullptr, nullptr};  // per-iteration completion events
  int step_cap = 0;                            // Strang steps w.step_sq holds
  std::vector<cudaEvent_t> step_events;        // phase boundaries of timed Strang steps
};

namespace kfbi {

// allocation helper: records the pointer for kfbi_destroy
template <typename T>
int dalloc(kfbi_handle* h, T** p, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    return KFBI_ERR_OOM;
  }
  h->allocations.push_back((void*)*p);
  h->device_bytes += count * sizeof(T);
  return KFBI_OK;
}

// ---- launchers implemented in the .cu files ----

// setup.cu
int setup_build(kfbi_handle* h, const kfbi_geometry* geom);

// dst.cu: box solve of r -> v on the padded grids
//  src     : optional user-layout float64 field added with weight alpha
//  corr    : optional compact corrections at the irregular nodes (float64)
//  out_user: optional user-layout float64 output  out = beta*v + gamma*aux
//  keep    : true = leave the solution in the padded work grid
struct SolveArgs {
  const double* src = nullptr;
  const float* src32 = nullptr;   // float32 source on the user layout (alpha not applied)
  double alpha = 1.0;
  const double* corr = nullptr;
  double* out_user = nullptr;
  const double* aux = nullptr;
  double beta = 1.0;
  double gamma = 0.0;
  double lambda = 0.0;
  bool keep = true;               // the x inverse pass also writes the padded work grid
  const float* aux32 = nullptr;   // float32 solves: out_user = beta v + aux32 (a padded float grid)
};
int box_solve64(kfbi_handle* h, const SolveArgs& a, double* work);
// the float64 box solve of the coupled pair (sources / corrections / outputs
// of the intracellular component in si, extracellular in se) on the padded
// grids wa, wb
int box_solve_coupled64(kfbi_handle* h, const SolveArgs& si, const SolveArgs& se, const Coupling& cp, double* wa,
                        double* wb);
int box_solve32(kfbi_handle* h, const SolveArgs& a, float* work);
// the same with float32 transforms (the 2 x 2 mode solve stays float64)
int box_solve_coupled32(kfbi_handle* h, const SolveArgs& si, const SolveArgs& se, const Coupling& cp, float* wa,
                        float* wb);
int dst_supported(int N);
int transform_pass(kfbi_handle* h, int precision, int pass, double lambda);
int make_tma_maps(kfbi_handle* h);

// ops.cu
int launch_correction(kfbi_handle* h, const double* x, double* corr);
// the same with an explicit row set (the coupled system's second component)
int launch_correction_t(kfbi_handle* h, const Tables& t, const double* x, double* corr);
int launch_limit64_t(kfbi_handle* h, const Tables& t, const double* grid, const double* x, const double* base, double sgn,
                     double* out);
int launch_limit_user_t(kfbi_handle* h, const Tables& t, const double* u, const double* x, const double* base,
                        double sgn, double* out);
int launch_rank_one_coupled(kfbi_handle* h, const double* psi, double* out, double sgn);
int launch_limit32_t(kfbi_handle* h, const Tables& t, const float* grid, const double* x, const double* base,
                     double sgn, double* out);
// float64 residual of the coupled system (both components) plus corrections
int launch_residual_coupled(kfbi_handle* h, const double* src_i, double a_i, const double* src_e, double a_e,
                            const double* corr_i, const double* corr_e, const double* ui, const double* ue,
                            double kappa, double* ri, double* re);
// V <- 2 ((a + b) - (c + d)) - V
int launch_midpoint4(kfbi_handle* h, double* V, const double* a, const double* b, const double* c, const double* d,
                     int64_t n);
// V <- 2 (a - b) - V
int launch_midpoint_diff(kfbi_handle* h, double* V, const double* a, const double* b, int64_t n);
// dst = src - mean over Omega of src
int launch_sub_mean(kfbi_handle* h, const double* src, double* dst);
int launch_spline(kfbi_handle* h, const double* psi, double* x);
int launch_limit64(kfbi_handle* h, const double* grid, const double* x, const double* base, double sgn, double* out);
int launch_limit32(kfbi_handle* h, const float* grid, const double* x, const double* base, double sgn, double* out);
int launch_scatter_grid(kfbi_handle* h, const double* corr, double* grid_user);
int launch_limit_user(kfbi_handle* h, const double* u, const double* x, const double* base, double sgn, double* out);
int launch_residual(kfbi_handle* h, const double* src, double alpha, const double* corr, const double* u, double lambda,
                    double* res);
// r = alpha*src + corr - L_h u (float32 result) for u held exactly by the
// padded float32 grid u32 (the output of a float32 solve) and by u64 on the
// user layout; float-float arithmetic away from the interface, float64 at
// irregular nodes
int launch_residual_ff_coupled(kfbi_handle* h, const double* src_i, double a_i, const double* src_e, double a_e,
                               const double* corr_i, const double* corr_e, const double* ui, const double* ue,
                               double kappa, float* ri, float* re);
int launch_residual_ff(kfbi_handle* h, const double* src, double alpha, const double* corr, const float* u32,
                       const double* u64, double lambda, float* res);
int launch_lincomb(kfbi_handle* h, double* y, double a, const double* x, double b, int64_t n);
// out += sgn <ds, psi> / |Gamma| (the rank-one term of the Poisson operator)
int launch_rank_one(kfbi_handle* h, const double* psi, double* out, double sgn);
// f = -lambda V + c I (V may be NULL)
int launch_stim_source(kfbi_handle* h, const double* V, double lambda, const double* I, double c, double* f,
                       int64_t n);
// ue = (S - sigma_i V) / (sigma_i + sigma_e) with zero mean over Omega
int launch_ue_S(kfbi_handle* h, const double* V, const double* S, double* ue);
int launch_padded_to_user(kfbi_handle* h, const double* padded, double* user);

// GMRES vector kernels (ops.cu)
int vec_dots(kfbi_handle* h, const double* V, int nvec, int ld, const double* w, double* out_dev);
int launch_gram(kfbi_handle* h, const double* H, int k, const double* g, double* G, double* b, double* gg);
int vec_update(kfbi_handle* h, double* w, const double* V, int nvec, int ld, const double* coef_dev, double sign);
int vec_axpby(kfbi_handle* h, double* y, double a, const double* x, double b, int n);
int vec_scale_by_norm(kfbi_handle* h, double* v, const double* w, const double* norm_dev, int n);
int vec_copy(kfbi_handle* h, double* dst, const double* src, int n);
int arnoldi_givens(kfbi_handle* h, double* small, int j, int ldh);
int arnoldi_step(kfbi_handle* h, double* V, int ld, double* wv, int j, int m, double gnorm, double tol);
int arnoldi_solve(kfbi_handle* h, double* small, int k, int ldh);

// mlp.cu
int mlp_warmstart(kfbi_mlp* m, cudaStream_t st, const double* psiF, const double* rF, const double* g,
                  const double* sq, const double* nodes, const double* normals, int M, double two_gamma,
                  double* out);
// training rows F [M][9] (raw features) and targets T [M] of one solve
int launch_train_rows(cudaStream_t st, const double* psi, const double* psiF, const double* rF, const double* g,
                      const double* sq, const double* nodes, const double* normals, int M, double two_gamma, float* F,
                      float* T);

int launch_react_fe(const kfbi_fhn* p, double k, double* V, double* w, int64_t n, cudaStream_t s);
// backward Euler of (V, w); with vV, vB: of the midpoint 2 (vV + vB) - V,
// formed in the same pass; fe_next: followed in the same pass by the forward
// Euler half step (same k) that opens the next Strang step
int launch_react_be(const kfbi_fhn* p, double k, double* V, double* w, int64_t n, int* err, cudaStream_t s,
                    const double* vV = nullptr, const double* vB = nullptr, bool fe_next = false);
int launch_ue(kfbi_handle* h, const double* V, double* ue);

}  // namespace kfbi
