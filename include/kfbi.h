/*
 * kfbi.h - C ABI of the GB300 kernel-free boundary integral (KFBI) library for
 * the FitzHugh-Nagumo bidomain equations (Gao, Cai, Henriquez, Ying,
 * "A kernel-free boundary integral method for the bidomain equations").
 *
 * Conventions for every entry point:
 *  - Returns KFBI_OK (0) or a positive KFBI_ERR_* code; never throws.  The
 *    message of the last failure on the calling thread is kfbi_last_error().
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; all
 *    other pointers are host pointers owned by the caller and only read during
 *    the call.  The library owns its workspace and tables (freed by
 *    kfbi_destroy).
 *  - Box grids cover [lo, hi]^dim with N intervals per axis, h = (hi - lo)/N,
 *    nodes x_k = lo + k h.  Grid fields are row-major [z][y][x] (x fastest),
 *    float64, contiguous.  With the Dirichlet box (kfbi_grid.box =
 *    KFBI_BOX_DIRICHLET) they hold the (N-1)^dim interior nodes k = 1..N-1
 *    and box-boundary nodes carry the value 0 of the interface problems
 *    (Section 5.1); with the Neumann box (KFBI_BOX_NEUMANN) they hold all
 *    (N+1)^dim nodes k = 0..N.
 *  - Interface-node vectors (densities psi, Neumann data g^N, limits) hold M
 *    float64 values in the order of kfbi_geometry.nodes.
 *  - Work is enqueued on kfbi_opts.stream (NULL = the legacy default stream).
 *    Entry points that iterate (GMRES, Strang steps) synchronise that stream
 *    to read residuals; all others only enqueue.
 */
#ifndef KFBI_H
#define KFBI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define KFBI_OK 0
#define KFBI_ERR_ARG 1            /* bad argument or unsupported size            */
#define KFBI_ERR_GEOMETRY 2       /* domain touches the box, stencil leaves grid */
#define KFBI_ERR_NOT_CONVERGED 3  /* outputs written, stats valid               */
#define KFBI_ERR_NAN 4            /* non-finite residual                         */
#define KFBI_ERR_CUDA 5           /* CUDA runtime failure                        */
#define KFBI_ERR_OOM 6            /* device allocation failed                    */
#define KFBI_ERR_NEWTON 7         /* backward-Euler Newton hit its iteration cap */

/* geometry kinds (domain Omega inside the box) */
#define KFBI_ELLIPSE2 1    /* params: a, b, cos, sin of the rotation          */
#define KFBI_ELLIPSOID3 2  /* params: a, b, c                                 */
#define KFBI_STAR3 3       /* params: A, B of r = A + B sin(3 theta) cos(2 phi) */
#define KFBI_SHELL3 4      /* params: outer a, b, c, inner a, b, c            */
#define KFBI_MESH3 5       /* no params: Omega is bounded by the closed triangle
                              mesh (nodes, tri) alone (Section 5.3, Example 4);
                              triangles wound counter-clockwise seen from
                              outside Omega; cube_t / cube_n / comp_* unused   */

/* surface-component point-location maps of 3-D cube-sphere meshes */
#define KFBI_MAP_RADIAL 0
#define KFBI_MAP_ELLIPSOID 1

/* box condition of the interface problems (kfbi_grid.box) */
#define KFBI_BOX_DIRICHLET 0 /* v = 0 on the box boundary; sine transforms          */
#define KFBI_BOX_NEUMANN 1   /* zero normal derivative on the box boundary, the box
                                Green's function of Section 4: mirrored ghost rows,
                                cosine (DCT-I) transforms; every precision,
                                lambda > 0 (no Green's function of the Poisson
                                operator), scalar problem only                    */

/* precision of the integral evaluations */
#define KFBI_FP64 0          /* all transforms and corrections in float64        */
#define KFBI_MIXED 1         /* float32 transforms inside GMRES, float64 Arnoldi,
                                residuals and outer refinement                   */
#define KFBI_MIXED_LEARNED 2 /* KFBI_MIXED + learned warm start of the density
                                (kfbi_set_warmstart)                             */
#define KFBI_FP32 3          /* kfbi_box_solve / kfbi_transform_pass only: plain
                                float32 transforms without refinement             */

#define KFBI_GMRES 0
#define KFBI_RICHARDSON 1

/* initial density of each diffusion solve in bidomain_step */
#define KFBI_WARM_PREVIOUS 0   /* the previous solve's density                */
#define KFBI_WARM_PROJECTION 1 /* least-squares combination of the last
                                  KFBI_HISTORY densities, chosen by their known
                                  images A psi_s, plus one step of the simple
                                  iteration (Section 4)                        */
#define KFBI_HISTORY 8

#define KFBI_MAX_COMP 4

/*
 * Interface description (Section 6: quasi-uniform interface nodes; Section
 * 5.3 / Fig. 1: three-dimensional surfaces given by a triangle mesh).
 *  nodes   [M][dim]       interface nodes.  2-D: counter-clockwise, equally
 *                         spaced in the curve parameter t_i = 2 pi i / M.
 *  tri     [n_tri][3]     3-D only: triangles of cube-sphere meshes of
 *                         resolution cube_n, one mesh per surface component,
 *                         triangle ((f n + j) n + i) 2 + half of component c
 *                         at comp_tri_offset[c] (face f, quad (i, j), half 0 =
 *                         (v_ij, v_i+1j, v_ij+1), half 1 = (v_i+1j, v_i+1j+1, v_ij+1)).
 *                         KFBI_MESH3: any closed, consistently wound manifold
 *                         mesh whose vertices are the nodes (vertex ring of a
 *                         triangle at most 16 points); it is the only
 *                         description of the surface.
 *  cube_t  [cube_n + 1]   equiangular face coordinates (-1 ... 1).
 */
typedef struct {
  int dim;
  int kind;
  double params[16];
  int n_nodes;
  const double* nodes;
  int n_tri;
  const int32_t* tri;
  int cube_n;
  const double* cube_t;
  int n_comp;
  int comp_map[KFBI_MAX_COMP];
  double comp_axes[KFBI_MAX_COMP][3];
  int comp_vert_offset[KFBI_MAX_COMP];
  int comp_n_vert[KFBI_MAX_COMP];
  int comp_tri_offset[KFBI_MAX_COMP];
} kfbi_geometry;

typedef struct {
  int dim;
  int N;
  double lo;
  double hi;
  int box;  /* KFBI_BOX_DIRICHLET or KFBI_BOX_NEUMANN */
} kfbi_grid;

typedef struct {
  int precision;   /* KFBI_FP64 / KFBI_MIXED / KFBI_MIXED_LEARNED            */
  int solver;      /* KFBI_GMRES / KFBI_RICHARDSON                           */
  double tol;      /* relative residual ||g - A psi|| / ||g||                */
  int restart;     /* GMRES restart length (<= 64)                           */
  int max_iter;    /* total operator applications allowed                    */
  double gamma;    /* Richardson parameter (0.8 in Section 7)               */
  void* stream;    /* cudaStream_t                                           */
  int warm;        /* KFBI_WARM_PREVIOUS / KFBI_WARM_PROJECTION (the learned
                      form always starts from the projection)               */
} kfbi_opts;

typedef struct {
  int iters;            /* operator applications inside the Krylov solver     */
  int outer;            /* outer refinement sweeps (mixed precision)          */
  int warmstart;        /* initial guess kept: 0 previous density or
                           projection, 1 learned                            */
  double rel_res;       /* solver's residual estimate ||r|| / ||g||           */
  double true_rel_res;  /* recomputed ||g^N - du^+/dn|| / ||g|| of the final
                           u = v_V + v_B(psi) (-1 where not computed)        */
  double init_rel_res;  /* residual of the initial guess                      */
  double ms;            /* host wall time of the call / step                  */
  /* bidomain_step only: device time of the phases of the step (CUDA events):
     both reaction half steps, the volume solve and g, the warm start, the
     boundary-integral solve, and the assembly of V (with the true residual;
     the float32 forms of the scalar step form the midpoint of V inside the
     backward-Euler pass, so there it counts as reaction time; within one
     call the forward half step of every step after the first runs in the
     previous step's backward pass and is timed with it) */
  double react_ms, rhs_ms, warm_ms, solve_ms, assemble_ms;
} kfbi_stats;

typedef struct {
  double H, theta, alpha, zeta, Cm, beta;   /* FitzHugh-Nagumo, Section 7 */
} kfbi_fhn;

typedef struct {
  int M;               /* interface nodes                       */
  int n_irregular;     /* irregular grid nodes                  */
  int n_crossings;     /* interface / grid-line crossings       */
  int n_inside;        /* grid nodes inside Omega               */
  size_t device_bytes; /* workspace and tables held on the GPU  */
  double lambda;       /* lambda = (2 / dt)(1/sigma_i + 1/sigma_e) of the
                          implicit-midpoint V problem with Cm beta = 1
                          (bidomain_step scales it by the kfbi_fhn's Cm beta) */
  int xy_fused;        /* 1: float32 3-D box solves take three passes (fused
                          x-y forward, z solve, fused x-y inverse)           */
} kfbi_info;

typedef struct kfbi_handle kfbi_handle;
typedef struct kfbi_mlp kfbi_mlp;

const char* kfbi_last_error(void);

/*
 * Setup (Section 6): classify the box nodes against the domain (bit-exact
 * level sets), list the irregular nodes and grid-line crossings, build the
 * correction and interpolation tables, sine-transform tables and workspace.
 * dt, sigma_i, sigma_e fix lambda = (2 Cm beta / dt)(1/sigma_i + 1/sigma_e) of
 * the implicit-midpoint diffusion step (Section 3, Eq. pde1) used by
 * bidomain_step with the FitzHugh-Nagumo parameters given there.
 * Errors: KFBI_ERR_ARG (unsupported N or dim), KFBI_ERR_GEOMETRY, KFBI_ERR_OOM.
 */
int kfbi_create(const kfbi_geometry* geom, const kfbi_grid* grid, double sigma_i, double sigma_e,
                double dt, const kfbi_opts* opts, kfbi_handle** out);
void kfbi_destroy(kfbi_handle* h);
int kfbi_query(kfbi_handle* h, kfbi_info* info);
int kfbi_set_opts(kfbi_handle* h, const kfbi_opts* opts);

/*
 * Neumann boundary value problem (Sections 4-5, Algorithm 1 with GMRES):
 *   Lap u - lambda u = f in Omega,  du/dn = gN on the boundary,
 * f given on every box node (its continuous extension, Section 5.1).
 * psi_dev: in = initial density (warm start), out = converged density.
 * u_dev:   out = u = v_V + v_B on every box node.
 * lambda = 0 (Poisson): A then has a one-dimensional null space and its range
 * is orthogonal to constants; every operator application uses the rank-one
 * modification A psi + <ds, psi>/|Gamma| (ds the boundary quadrature weights:
 * 2-D half the two chord lengths at a node, 3-D a third of the incident
 * triangle areas), which has the same solutions for compatible data and
 * absorbs the small incompatibility of discrete data.
 * Returns KFBI_ERR_NOT_CONVERGED (outputs still written) if max_iter is hit.
 */
int kfbi_solve_neumann(kfbi_handle* h, double lambda, const double* f_dev, const double* gN_dev,
                       double* u_dev, double* psi_dev, kfbi_stats* stats);

/*
 * nsteps Strang steps (Section 3): forward-Euler reaction over dt/2, implicit
 * midpoint diffusion over dt (backward Euler over dt/2 for w, then
 * V = 2 w - V), backward-Euler reaction over dt/2 (Newton, |dV| < 1e-10, cap 50).
 * V_dev, w_dev: in/out state on all box nodes; ue_dev (may be NULL): out
 * extracellular potential with zero mean over Omega.  The density of the last
 * diffusion solve is kept in the handle and warm-starts the next one.
 * per_step: nsteps entries or NULL.
 */
int bidomain_step(kfbi_handle* h, const kfbi_fhn* p, double* V_dev, double* w_dev, double* ue_dev,
                  int nsteps, kfbi_stats* per_step);
/* bidomain_step with the extracellular stimulus of a virtual electrode
 * (Section 7): istim_dev (user layout, float64) is I_stim on every interior
 * node, constant in time.  The isotropic elimination of Eq. pde1 gives
 *   Lap V - lambda V = -lambda V^n + beta I / sigma_e      (V problem),
 *   Lap S = -beta I,  S = sigma_i Phi_i + sigma_e Phi_e     (S problem),
 * both with homogeneous Neumann data.  The S problem (lambda = 0, with the
 * rank-one modification described at kfbi_solve_neumann) is solved once per
 * call; ue_dev (optional) receives Phi_e = (S - sigma_i V)/(sigma_i +
 * sigma_e) with zero mean over Omega.  NULL istim_dev is bidomain_step.  The
 * first stimulated call on a handle allocates two grid-sized work arrays.    */
int kfbi_bidomain_step_stim(kfbi_handle* h, const kfbi_fhn* p, const double* istim_dev, double* V_dev,
                            double* w_dev, double* ue_dev, int nsteps, kfbi_stats* per_step);

/* ------------------------------------------------------------------
 * Anisotropic coupled system (Section 5.2: fibres along the axes, diagonal
 * conductivity tensors D_i = diag(D_i[0..dim-1]), D_e likewise; Eq. pde1).
 * The backward-Euler half step of the diffusion is the vector Neumann
 * problem
 *   div(D_i grad Phi_i) - kappa (Phi_i - Phi_e) = f_i,
 *   div(D_e grad Phi_e) + kappa (Phi_i - Phi_e) = f_e,
 *   n.D_i grad Phi_i = gN_i,  n.D_e grad Phi_e = gN_e,
 * solved by the KFBI method with the density pair psi = (psi_i, psi_e)
 * (2M doubles, psi_i first): per-component corrections with the conormal
 * jump relations of the component's D, a box solve by sine transforms with a
 * 2 x 2 solve per mode, conormal limits n.D grad v^+.  Constants (c, c) solve
 * the homogeneous problem, so every operator application adds the rank-one
 * term (1, 1) <(ds, ds), psi> / (2 |Gamma|) (ds as at kfbi_solve_neumann);
 * Phi_i and Phi_e are then fixed up to that common constant's choice, their
 * difference is unique.  opts.precision KFBI_FP64 (float64 throughout) or
 * KFBI_MIXED (float32 transforms inside GMRES, float64 Arnoldi, and
 * refinement of the coupled residual, its first round in float-float
 * arithmetic, for g, the outer residuals and the final potentials).  The
 * 2 x 2 mode solve multiplies by three factors per mode, computed in float64
 * once per kappa into a device table of 3 N^dim values of the transform's
 * type that the handle allocates on first use and frees at kfbi_destroy.
 * Dirichlet box only.
 * ------------------------------------------------------------------ */
/* Setup as kfbi_create for the coupled system; D_i, D_e: dim positive
 * conductivities each (host).  bidomain_step and kfbi_bidomain_step_stim on
 * this handle run the Strang step with the coupled diffusion (kappa = 2 Cm
 * beta / dt, f = (-kappa V, kappa V - beta I_stim), warm start: the previous
 * density pair, or with opts.warm = KFBI_WARM_PROJECTION the history
 * projection of the density pairs; V <- 2 (Phi_i - Phi_e) - V); their ue_dev
 * receives the last solve's Phi_e (the midpoint level t^n + dt/2) with zero
 * mean over Omega.                                                           */
int kfbi_create_coupled(const kfbi_geometry* geom, const kfbi_grid* grid, const double* D_i, const double* D_e,
                        double dt, const kfbi_opts* opts, kfbi_handle** out);
/* The coupled Neumann problem: fi_dev, fe_dev on every box node (continuous
 * extensions), gNi_dev, gNe_dev [M]; psi_dev [2M] in: initial guess, out:
 * density pair; phi_i_dev, phi_e_dev: out on every box node.  stats as at
 * kfbi_solve_neumann (true_rel_res includes the rank-one term).            */
int kfbi_solve_coupled(kfbi_handle* h, double kappa, const double* fi_dev, const double* fe_dev,
                       const double* gNi_dev, const double* gNe_dev, double* phi_i_dev, double* phi_e_dev,
                       double* psi_dev, kfbi_stats* stats);
/* (v_i, v_e) = L_h^{-1} (r_i, r_e) of the coupled 5/7-point operator with
 * zero Dirichlet data on the box (Eq. FDE, float64).                       */
int kfbi_box_solve_coupled(kfbi_handle* h, double kappa, const double* ri_dev, const double* re_dev, double* vi_dev,
                           double* ve_dev);
/* out [2M] = A psi [2M] of the coupled boundary integral equation (conormal
 * limits of the single layer, plus the rank-one term).                     */
int kfbi_apply_A_coupled(kfbi_handle* h, double kappa, const double* psi_dev, double* out_dev);

/* ------------------------------------------------------------------
 * Step-level entry points (one per row of the hot path), used for parity
 * checks and benchmarks.  All act on the handle's geometry and grid.
 * ------------------------------------------------------------------ */

/* Export setup results to host buffers (NULL to skip any):
 * inside [(N-1)^dim] uint8; irregular [n_irregular] int32 flat indices
 * (increasing); crossing_axis/crossing_lo [n_crossings] int32 and crossing_z
 * [n_crossings] float64, sorted by (axis, lower node); center [M][dim] int32
 * 1-based node indices; sign [M][dim] int8.                                  */
int kfbi_export_setup(kfbi_handle* h, uint8_t* inside, int32_t* irregular, int32_t* crossing_axis,
                      int32_t* crossing_lo, double* crossing_z, int32_t* center, int8_t* sign);

/* Export the precomputed linear rows of the hot path (NULL to skip any):
 * node_wn [M][P] Taylor weights of dv/dn on the stencil values (P = 6 / 10);
 * node_cnt [M], node_pid [M][17], node_w [M][17]: each node's jump row on the
 * density vector (psi in 3-D, [psi; spline moments] in 2-D);
 * cross_cnt [n_crossings], cross_pid/cross_wlo/cross_whi [n_crossings][16]:
 * each crossing's correction row for its lower and upper end node.          */
int kfbi_export_tables(kfbi_handle* h, double* node_wn, int32_t* node_cnt, int32_t* node_pid, double* node_w,
                       int32_t* cross_cnt, int32_t* cross_pid, double* cross_wlo, double* cross_whi);

/* Box solve (Sections 5.2-5.3): v = L_h^{-1} r, 5/7-point operator with the
 * handle's box condition (zero Dirichlet data by sine transforms, or the
 * Neumann box's mirrored ghost rows by cosine transforms).  precision
 * KFBI_FP64 (float64 transforms), KFBI_MIXED / KFBI_MIXED_LEARNED (float32
 * transforms refined by one round of the float64 residual, two when the
 * handle's tolerance is below 1e-9: float64-accurate) or KFBI_FP32 (float32
 * transforms only).                                                         */
int kfbi_box_solve(kfbi_handle* h, int precision, double lambda, const double* r_dev, double* v_dev);

/* Irregular-node correction (Section 5.3, Eq. correct): rhs_dev (grid, fully
 * written) = 0 at regular nodes, summed corrections from the jumps of the
 * single layer with density psi at irregular nodes.                          */
int kfbi_correction(kfbi_handle* h, const double* psi_dev, double* rhs_dev);

/* Interface limit (Section 5.4): out[i] = dv^+/dn at node i from the Taylor
 * system, with the single-layer jumps of psi_dev (NULL = no jumps).          */
int kfbi_interface_limit(kfbi_handle* h, const double* v_dev, const double* psi_dev, double* out_dev);

/* Matrix-vector product of the boundary integral equation (Algorithm 1):
 * out = A psi = dv_B^+/dn.                                                   */
int kfbi_apply_A(kfbi_handle* h, int precision, double lambda, const double* psi_dev, double* out_dev);

/* Right-hand side g = gN - dv_V^+/dn with v_V the box solve of f.           */
int kfbi_rhs_g(kfbi_handle* h, double lambda, const double* f_dev, const double* gN_dev, double* g_dev);

/* GMRES / Richardson on A psi = g alone (tol = 0 runs exactly max_iter
 * applications).                                                             */
int kfbi_solve_bie(kfbi_handle* h, double lambda, const double* g_dev, double* psi_dev, kfbi_stats* stats);

/* ------------------------------------------------------------------
 * Learned warm start (the workload's mixed + learned form; not in the paper).
 * A point-wise network on the interface nodes reads 9 raw features per node,
 *   (psi_F / rms(psi_F), r_F / rms(r_F), g / rms(g), x, y, z, n_x, n_y, n_z),
 * with psi_F the history projection (KFBI_WARM_PROJECTION), r_F = g - A psi_F
 * its residual, g the right-hand side of the solve and rms the root mean
 * square over the nodes; they are normalised by norm = [mean[9], std[9],
 * out_mean, out_std], pass 4 hidden layers of width 128 with SiLU, and give
 * an output o.  The initial density is
 *   psi_L = psi_F + 2 gamma r_F + rms(r_F) (out_std o + out_mean).
 * Parameters (float32, packed W0[128][9], b0[128], W1[128][128], b1, W2, b2,
 * W3, b3, W4[1][128], b4[1]) are kept as float32 masters with bfloat16 copies
 * for the tensor-core products (float32 accumulation).  Training uses the
 * loss 0.5 mean (o - t)^2 on the normalised targets t = (T - out_mean) /
 * out_std of raw targets T (kfbi_training_rows) and Adam (0.9, 0.999, 1e-8).
 * ------------------------------------------------------------------ */
int kfbi_mlp_num_params(void);
/* params_host [kfbi_mlp_num_params()], norm_host [20]; max_batch rows per
 * call; work on `stream`.                                                    */
int kfbi_mlp_create(const float* params_host, const float* norm_host, int max_batch, void* stream, kfbi_mlp** out);
void kfbi_mlp_destroy(kfbi_mlp* m);
int kfbi_mlp_get(kfbi_mlp* m, float* params_host);
/* o_dev[B] = network output for raw features F_dev [B][9] (float32).        */
int kfbi_mlp_forward(kfbi_mlp* m, const float* F_dev, int B, float* o_dev);
/* loss and (optionally) the gradient of every parameter to host memory, for
 * raw features F_dev [B][9] and raw targets T_dev [B] (device, float32).     */
int kfbi_mlp_grad(kfbi_mlp* m, const float* F_dev, const float* T_dev, int B, float* loss_host, float* grad_host);
/* one forward + backward + Adam step with learning rate lr.                 */
int kfbi_mlp_train_step(kfbi_mlp* m, const float* F_dev, const float* T_dev, int B, float lr, float* loss_host);
/* Layer values of the training path, for element-wise checks of every
 * kernel of the network (no counterpart in the paper): the forward pass of
 * kfbi_mlp_grad on B raw rows F_dev [B][9] gives z_dev [4][B][128], the
 * pre-activations z_l = bf16(a_l) bf16(W_l)^T + b_l of the hidden layers
 * l = 0..3, and o_dev [B]; with raw targets T_dev its backward pass gives
 * d_dev [4][B][128], dL/dz_l of the hidden layers in the order l = 3..0, and
 * d4_dev [B] = dL/do.  Outputs are device float32 and may be NULL;
 * synchronises the network's stream.                                        */
int kfbi_mlp_layers(kfbi_mlp* m, const float* F_dev, const float* T_dev, int B, float* z_dev, float* o_dev,
                    float* d_dev, float* d4_dev);
/* Normalisation vector of a training set (norm_host [20]): per feature the
 * mean and sample standard deviation of F_dev [n][9], then those of T_dev
 * [n]; a spread below 1e-12 (features) or 1e-30 (targets) becomes 1.  Work
 * on `stream`, synchronised; allocates 160 bytes of device scratch.          */
int kfbi_mlp_fit_norm(const float* F_dev, const float* T_dev, int n, void* stream, float* norm_host);
/* Attach (or detach with NULL) a network to a 3-D handle.  With precision
 * KFBI_MIXED_LEARNED, bidomain_step then starts each diffusion solve from
 *   psi_L = psi_F + 2 gamma r_F + rms(r_F) * net(psi_F/rms, r_F/rms, g/rms,
 *                                                 x, n),
 * psi_F the history projection (KFBI_WARM_PROJECTION) and r_F its residual,
 * and keeps psi_L only when its float64-accurate residual ||g - A psi_L|| is
 * below ||r_F||; otherwise it starts from psi_F, whose residual is never
 * above that of the previous density (which lies in the projection's span).
 * Network input rows are (psi_F, r_F, g^n) scaled by their root mean
 * squares, then the node and its unit normal; the output is the correction
 * in units of rms(r_F), with the normalisation of kfbi_mlp_create.          */
int kfbi_set_warmstart(kfbi_handle* h, kfbi_mlp* m);
/* After a Strang step: psi_dev <- psi^n, psi_prev_dev <- psi^{n-1} and
 * g_dev <- g^n of the last diffusion solve (each may be NULL).               */
int kfbi_get_densities(kfbi_handle* h, double* psi_dev, double* psi_prev_dev, double* g_dev);
/* Restore the density history saved by kfbi_get_densities (checkpoint /
 * resume): n_solves is the number of diffusion solves the history stands for
 * (0 clears it).  With the same state (V, w) a resumed run with the
 * previous-density start repeats the uninterrupted one bit for bit.  It
 * empties the projection history; runs with KFBI_WARM_PROJECTION (or the
 * learned form) resume through kfbi_get_history / kfbi_set_history instead.  */
int kfbi_set_densities(kfbi_handle* h, const double* psi_dev, const double* psi_prev_dev, const double* g_dev,
                       int n_solves);
/* The density history of the projection warm start: KFBI_HISTORY slots of
 * M doubles each (psi and its image A psi: with the float32 forms g - r, r the
 * solve's final float64-accurate residual; with float64 the right-hand side
 * g, equal to A psi to the tolerance; the density of solve s sits in slot
 * s mod KFBI_HISTORY) and the number of solves it stands for.  get
 * copies out (device buffers of KFBI_HISTORY*M doubles, n_solves on the
 * host); set restores them (checkpoint / resume).                          */
int kfbi_get_history(kfbi_handle* h, double* psi_hist_dev, double* g_hist_dev, int* n_solves);
int kfbi_set_history(kfbi_handle* h, const double* psi_hist_dev, const double* g_hist_dev, int n_solves);
/* After a projection (or learned) step: the projected density psi_F and its
 * residual r_F = g - A psi_F (known without an operator application from the
 * history's images), M doubles each, device.                                */
int kfbi_get_projection(kfbi_handle* h, double* psiF_dev, double* rF_dev);
/* After a Strang step: the initial density its diffusion solve started from,
 * before the residual judge (psi_L of the learned form, psi_F + 2 gamma r_F
 * of the projection form, the previous density otherwise), M doubles.      */
int kfbi_get_warm_guess(kfbi_handle* h, double* psi0_dev);
/* Training rows of the learned warm start from the last Strang step of a 3-D
 * handle run with KFBI_WARM_PROJECTION (or the learned form): F_dev [M][9]
 * the network's raw input rows of that step's projection (the features
 * above) and T_dev [M] the raw target (psi - psi_F - 2 gamma r_F) / rms(r_F),
 * psi the converged density; float32, device, enqueued on the handle's
 * stream.                                                                    */
int kfbi_training_rows(kfbi_handle* h, float* F_dev, float* T_dev);

/* One pass of the box solver on the handle's padded work grid, for timing
 * the transform kernels in isolation: pass 0 = x forward (no right-hand
 * side), 1 = y forward, 2 = z solve (forward, spectral divide, inverse; the
 * y solve in 2-D), 3 = x inverse; with kfbi_info.xy_fused also 4 = fused x-y
 * forward and 5 = fused x-y inverse (KFBI_MIXED).  precision KFBI_FP64 or
 * KFBI_MIXED.  The grid content is arbitrary afterwards.                     */
int kfbi_transform_pass(kfbi_handle* h, int precision, int pass, double lambda);

/* Self-test of the bounded waits of the TMA-fed transform kernels (no
 * counterpart in the paper): one block polls an mbarrier that nothing ever
 * completes, with the same wait as those kernels, capped at `polls` polls
 * (1 .. 2^20).  *timed_out = 1 when the cap ended the wait and raised the
 * timeout flag (the expected outcome); *ms (optional) is the kernel time.
 * Allocates a 4-byte flag.                                                   */
int kfbi_selftest_bounded_wait(int polls, int* timed_out, double* ms);

/* Number of kernels this library has launched in the process so far
 * (instrumentation; every launch site adds its kernel count).                */
int64_t kfbi_launch_count(void);

/*
 * Box solve for callers that cannot allocate device memory (the paper has no
 * counterpart).  Same operation and result as kfbi_box_solve with precision
 * KFBI_FP64 -- v = L_h^{-1} r on the (N-1)^dim interior nodes of [lo, hi]^dim
 * with zero Dirichlet data -- but without a handle and without any device
 * allocation: some callers run where every byte of device memory belongs to a
 * pool or arena they do not control, or where allocation after start-up is
 * forbidden, so neither they nor a library called by them may call
 * cudaMalloc.  The padded work grid and the transform tables live in one
 * static device array of KFBI_NOALLOC_MAX_POINTS + 2560 doubles (about 2 MiB)
 * that every GPU loading this library holds until the process exits.
 *  - N^dim must not exceed KFBI_NOALLOC_MAX_POINTS (3-D: N <= 64; 2-D:
 *    N <= 512; N in 8, 16, 32, 64, 128, 256, 384, 512), else KFBI_ERR_ARG.
 *  - The first call on a device (with that device current) looks up the
 *    array's device address with cudaGetSymbolAddress; make that first call
 *    before any stream capture.
 *  - Every call shares the array, which keeps the last call's contents, so
 *    calls that overlap on the GPU (other streams, other host threads using
 *    the same device) race and must be serialised by the caller.
 *  - r_dev, v_dev: caller-owned device fields, float64, (N-1)^dim, [z][y][x].
 *  - Work is enqueued on `stream`; the call does not synchronise.
 */
#define KFBI_NOALLOC_MAX_POINTS 262144
int kfbi_box_solve_noalloc(int dim, int N, double lo, double hi, double lambda, const double* r_dev,
                           double* v_dev, void* stream);

/* Pointwise FitzHugh-Nagumo half steps (Section 3, Eqs. ode1/ode2) over n
 * values: forward Euler (k = dt/2) and backward Euler with Newton.  The
 * backward step returns KFBI_ERR_NEWTON if any node hit the iteration cap.    */
int kfbi_react_fe(const kfbi_fhn* p, double k, double* V_dev, double* w_dev, int64_t n, void* stream);
int kfbi_react_be(const kfbi_fhn* p, double k, double* V_dev, double* w_dev, int64_t n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* KFBI_H */
