/*
 * dg.h -- C ABI of the GB300 (sm_103a) matrix-free DG TR-BDF2 projection
 * solver for the incompressible Navier-Stokes equations in artificial
 * compressibility form, after Orlando, Della Rocca, Barbante, Bonaventura,
 * Parolini, "An efficient and accurate implicit DG solver for the
 * incompressible Navier-Stokes equations" (arXiv 2107.07776).
 *
 * Conventions (all entry points):
 *  - Every field pointer is a caller-owned DEVICE pointer on the current CUDA
 *    device unless its comment says "host".  The library never frees caller
 *    memory; it owns and frees its own scratch.
 *  - Velocity fields are structure-of-arrays [component][cell][node], pressure
 *    fields [cell][node].  Cells are lexicographic (x fastest) over the
 *    structured box; nodes are lexicographic (x fastest) over the
 *    Gauss-Legendre points of [0,1]^d: k+1 per direction for the velocity
 *    space Q_k and k per direction for the pressure space Q_{k-1} (Section 3).
 *  - Work is enqueued on the caller's stream (`stream` is a cudaStream_t, NULL
 *    = legacy default stream).  Calls that return iteration counts or
 *    residuals synchronise that stream before returning.  The solver calls
 *    (dg_solve_stage, trbdf2_step, dg_solver_set_history) run on the solver's
 *    own non-blocking stream instead: each first waits for the work enqueued
 *    on the caller's stream -- the one named by dg_solver_set_stream, by
 *    default the legacy default stream (and so every blocking stream) -- and
 *    synchronises before it returns.  Kernels are launched with programmatic
 *    dependent launch on non-default streams (DG_PDL=0 in the environment
 *    turns it off).
 *  - Errors come back as dg_status; dg_last_error() gives a message for the
 *    calling thread.  No C++ exception crosses the ABI and no kernel traps:
 *    device-side failures set a device status word checked at call end.
 *  - Velocity and pressure pointers passed to one call must not alias each
 *    other unless stated.
 */
#ifndef DG_H
#define DG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_EINVAL = 1,        /* bad argument (null pointer, size, option) */
  DG_ECUDA = 2,         /* CUDA runtime error (message in dg_last_error) */
  DG_ENOMEM = 3,        /* device or host allocation failed */
  DG_ENOCONV = 4,       /* Krylov solve hit max_iter above tolerance */
  DG_EBREAKDOWN = 5,    /* non-finite residual or Krylov breakdown */
  DG_ETIMEOUT = 6,      /* solve exceeded its wall-clock limit */
  DG_EUNSUPPORTED = 7   /* valid request that the library does not implement */
} dg_status;

typedef struct dg_mesh dg_mesh;     /* geometry, 1D tables, MG hierarchy */
typedef struct dg_solver dg_solver; /* Krylov/MG workspaces, history, guess net */

enum { DG_MAP_CARTESIAN = 0, DG_MAP_GRADED_TANH = 1, DG_MAP_PERTURBED_SIN = 2 };

/* Structured box mesh of hexahedra (quadrilaterals for dim = 2), Section 3.
 *  n_cells[a]   cells along axis a (n_cells[2] ignored in 2D), >= 1
 *  lo, hi       box corners
 *  periodic[a]  1: periodic in axis a; 0: Dirichlet velocity walls with
 *               homogeneous Neumann pressure (Section 2, Eq. ns_artcomp)
 *  degree_u     velocity degree k (2..4); pressure degree k-1
 *  map          DG_MAP_CARTESIAN; DG_MAP_GRADED_TANH with map_param[a] = beta
 *               per axis (vertex x = lo + (hi-lo)(1 - tanh(beta(1-2 eta))/
 *               tanh(beta))/2, beta = 0: uniform); DG_MAP_PERTURBED_SIN with
 *               map_param[0] = A (every vertex shifted by
 *               A (hi-lo) prod_a sin(2 pi eta_a), trilinear cells). */
typedef struct {
  int32_t dim;
  int32_t n_cells[3];
  double lo[3], hi[3];
  int32_t periodic[3];
  int32_t degree_u;
  int32_t map;
  double map_param[3];
} dg_mesh_desc;

/* Build geometry, penalties (sigma = (k+1)^2 |Gamma|/|K| for velocity,
 * k^2 |Gamma|/|K| for pressure: Eq. penconst1 and its pressure analogue read
 * with face measure over cell volume) and the 1D tables on the current
 * device.  `stream` orders the uploads.  *out owns device memory until
 * dg_mesh_destroy.  Trilinear (DG_MAP_PERTURBED_SIN) meshes also hold the
 * per-point metric terms of their cells, computed once here in FP64 (with
 * FP32 copies): per velocity node the diffusion metric, mass weight and
 * inverse-Jacobian weights (16 doubles in 3D), per pressure node 7, per face
 * point the surface weight, normal and normal-derivative coefficients of
 * both sides (10 velocity, 7 pressure).  DG_EUNSUPPORTED for map/degree
 * combinations not built. */
dg_status dg_mesh_create(const dg_mesh_desc* desc, void* stream, dg_mesh** out);
void dg_mesh_destroy(dg_mesh* mesh);

/* Sizes: cells, velocity DoFs (all components), pressure DoFs.  Any output
 * pointer (host) may be NULL. */
dg_status dg_mesh_info(const dg_mesh* mesh, int64_t* n_cells, int64_t* n_dofs_u,
                       int64_t* n_dofs_p);

/* Physical coordinates of the nodes of field 0 (velocity nodes, one
 * component's worth) or 1 (pressure nodes): xyz [dim][cell][node], double,
 * device.  Synchronous. */
dg_status dg_mesh_node_coords(const dg_mesh* mesh, int32_t field, double* xyz, void* stream);

/* Coefficients of the momentum operator of one TR-BDF2 stage (Section 3,
 * Eqs. weakform_u_1 / weakform_u_2):
 *   mass * M + visc * A + adv * C(ubar)
 * stage 1: mass = 1/(gamma dt), visc = 1/(2 Re), adv = 1/2
 * stage 2: mass = 1/((1-gamma) dt), visc = a33/Re, adv = a33. */
typedef struct {
  double mass, visc, adv;
} dg_momentum_coeffs;

/* dst = (mass M + visc A + adv C(ubar)) src for every velocity component
 * (the operator is the same scalar operator per component, Section 3):
 * M mass matrix, A the SIP form a_u (Eq. bilin_diff, interior and wall
 * faces), C the local Lax-Friedrichs form c (Eq. trilinear) with the
 * advecting field ubar.  Homogeneous: Dirichlet data enter only through
 * dg_rhs_momentum.  src, ubar, dst: n_dofs_u doubles; dst must not alias
 * src or ubar.  FP64 throughout. */
dg_status dg_apply_momentum(dg_mesh* mesh, const dg_momentum_coeffs* co, const double* ubar,
                            const double* src, double* dst, void* stream);

/* Arithmetic of the FP64 operator applies of this mesh (storage stays FP64):
 * mode 0 (default) float-float -- every number as the unevaluated sum of two
 * FP32 values (48-bit significand, FP32 exponent range) computed on the FP32
 * pipes, which GB300 issues at about 61x its FP64 rate; mode 1 native FP64.
 * The environment variable DG_FP64_NATIVE=1 sets mode 1 for new meshes. */
dg_status dg_mesh_set_fp64_arith(dg_mesh* mesh, int32_t mode);

/* FP32 variant of dg_apply_momentum (multigrid smoothing and mixed-precision
 * preconditioning); same layout with float. */
dg_status dg_apply_momentum_f32(dg_mesh* mesh, const dg_momentum_coeffs* co, const float* ubar,
                                const float* src, float* dst, void* stream);

/* dst = (alpha M^p + K) src: the pressure Helmholtz operator of Eqs.
 * helmholtz_1 / helmholtz_2 (K the SIP form a_p of Eq. weakform_p_1, interior
 * faces only; homogeneous Neumann walls add nothing).  alpha =
 * 1/(c^2 gamma^2 dt^2) (stage 1) or 1/(c^2 (1-gamma)^2 dt^2) (stage 2).
 * src, dst: n_dofs_p doubles, no aliasing. */
dg_status dg_apply_poisson(dg_mesh* mesh, double alpha, const double* src, double* dst,
                           void* stream);

/* FP32 variant of dg_apply_poisson. */
dg_status dg_apply_poisson_f32(dg_mesh* mesh, double alpha, const float* src, float* dst,
                               void* stream);

/* Autotuner (a project addition): times the candidate tile shapes (cells per
 * CTA) of this mesh's operator kernels -- pressure Helmholtz, momentum with
 * and without advection, FP64 and FP32 -- with CUDA events on `stream` and
 * keeps the fastest for later applies.  Candidates: cells per CTA, a
 * register cap, the face-once form (every face evaluated once into a
 * per-mesh flux scratch, then the cells: a different rounding order, the
 * same result to FP64 rounding) and, for the 3D pressure operator on two
 * points per direction in FP32 and float-float arithmetic, the
 * tensor-product form (1D SIP blocks tabulated per axis cell, one thread per
 * cell; again the same result up to rounding order).  A mesh using
 * the face-once form shares that scratch between its applies, so applies
 * on one tuned mesh from different streams must not overlap.
 * Multigrid levels built afterwards from a tuned mesh are tuned too.
 * Trilinear meshes time the general kernel's three tile shapes (half,
 * default and double the cells per CTA) instead.  Results are cached in a JSON file (path DG_TUNE_CACHE, default
 * $HOME/.cache/dgns_autotune.json when that directory exists; "off"
 * disables it), keyed by device name, compute capability, library build and
 * mesh signature: a hit restores the choices without timing.  Allocates
 * temporary device buffers; synchronous. */
dg_status dg_autotune(dg_mesh* mesh, void* stream);

/* Sets the operator kernels' tile variant of this mesh by hand (0..7, the
 * candidates listed in dg_autotune's report: 0-2 cells per CTA half /
 * default / double, 3-4 default with 96 / 80 registers, 5-6 face-once
 * capped at 72 registers (6: every component's volume sums between the
 * same two barriers), 7 the Q1 tensor-product form (two threads per Q1
 * cell with native FP64 arithmetic) -- 3D scalar operators without
 * advection on two points per direction, in every precision; other
 * operators run variant 1 instead) for every operator and
 * precision; a face-once variant allocates the mesh's flux scratch.
 * Trilinear meshes take 0-2 as the general kernel's tile shapes (half,
 * default, double the cells per CTA) and run 1 for the others. */
dg_status dg_mesh_set_variant(dg_mesh* mesh, int32_t variant);

/* JSON list of the tuning choices and timings of a mesh ("[]" if untuned),
 * written to buf (host, size bytes). */
dg_status dg_autotune_report(const dg_mesh* mesh, char* buf, int64_t size);

/* ---------------------------------------------------------------------
 * Stage right-hand sides and updates (once per stage; Sections 2-3).
 * ------------------------------------------------------------------- */

/* Explicit part of F_u (Eq. rhs1 and its stage-2 analogue) plus the mass
 * term and data, for every velocity component:
 *   rhs = mass * M u_mass
 *       + sum_{t < n_terms} [ visc[t] * E_v w[t] + adv[t] * E_a(wbar[t]) w[t] ]
 *       + G p
 *       + dir_visc * B_v uD + dir_adv * B_a(ubar) uD      (uD != NULL)
 *       + M f                                              (f != NULL)
 * E_v: unpenalised viscous form -int grad w : grad v + sum_E {{grad w}}:<<v>>
 * E_a: central advective form +int (w x wbar) : grad v - sum_E {{w x wbar}}:<<v>>
 * G:   DG pressure gradient int p div v - sum_E {{p}} [[v]]
 * B_v, B_a: boundary data terms of Eq. rhs1 (SIP and LF with the trace of uD;
 *        the LF speed on walls is |ubar . n|, the paper's mirror-state speed
 *        for tangential data u_D . n = 0, see dg_step_params).
 * All faces of the skeleton take part in E_v, E_a, G (boundary averages are
 * interior traces).  All fields device pointers; u_mass, w[t], wbar[t], uD,
 * ubar, f have n_dofs_u doubles, p has n_dofs_p; rhs must alias none. */
typedef struct {
  double mass;
  const double* u_mass;
  int32_t n_terms;              /* 0, 1 or 2 */
  double visc[2], adv[2];
  const double* w[2];
  const double* wbar[2];
  const double* p;              /* NULL: no pressure gradient */
  const double* uD;             /* NULL: no Dirichlet data */
  double dir_visc, dir_adv;
  const double* ubar;           /* advecting field of the stage (LF speed of B_a) */
  const double* f;              /* NULL: no forcing */
} dg_momentum_rhs;

dg_status dg_rhs_momentum(dg_mesh* mesh, const dg_momentum_rhs* desc, double* rhs,
                          void* stream);

/* u_tilde = M^{-1} P p for every velocity component: the projection of the
 * broken pressure gradient into V_h (Section 3, matrix P).  p: n_dofs_p,
 * u_tilde: n_dofs_u. */
dg_status dg_project_gradient(dg_mesh* mesh, const double* p, double* u_tilde, void* stream);

/* rhs = alpha M^p p_old + (1/tau) sum_c D_c uss_c: right-hand side of the
 * pressure Helmholtz equation (Eqs. helmholtz_1, weakform_p_1), D the DG
 * divergence int u.grad q - sum_E {{u}}.[[q]] over all faces. */
dg_status dg_rhs_pressure(dg_mesh* mesh, double alpha, double tau, const double* uss,
                          const double* p_old, double* rhs, void* stream);

/* Diagonal of mass M + visc A + adv C(ubar) (Jacobi preconditioner of the
 * momentum systems, Section 4) for one scalar component: n_dofs_u/dim. */
dg_status dg_momentum_diagonal(dg_mesh* mesh, const dg_momentum_coeffs* co, const double* ubar,
                               double* diag, void* stream);

/* Diagonal of alpha M^p + K: n_dofs_p. */
dg_status dg_poisson_diagonal(dg_mesh* mesh, double alpha, double* diag, void* stream);

/* ---------------------------------------------------------------------
 * Solvers and the TR-BDF2 step.
 * ------------------------------------------------------------------- */
enum { DG_SYS_MOMENTUM = 0, DG_SYS_HELMHOLTZ = 1 };
enum { DG_PC_NONE = 0, DG_PC_JACOBI = 1, DG_PC_MG_FP64 = 2, DG_PC_MG_FP32 = 3 };
enum { DG_GUESS_ZERO = 0, DG_GUESS_EXTRAP = 1, DG_GUESS_LEARNED = 2, DG_GUESS_GIVEN = 3 };

typedef struct {
  int32_t system;       /* DG_SYS_* */
  double tol_rel;       /* stop when ||r|| <= tol_rel ||b|| */
  int32_t max_iter;     /* iterations (GMRES: total inner iterations) */
  int32_t restart;      /* GMRES restart length (momentum) */
  int32_t precond;      /* DG_PC_*: momentum takes NONE/JACOBI, Helmholtz any */
  int32_t guess;        /* DG_GUESS_* */
  double timeout_s;     /* wall-clock limit, <= 0: none */
  int32_t mg_degree;    /* Chebyshev degree of the multigrid smoother (pre and
                           post, every level); <= 0: the default, 5 */
} dg_solve_opts;

typedef struct {
  int32_t iterations;
  double res0, res_final;   /* ||b - A x0||, ||b - A x|| (2-norms) */
  int32_t status;           /* dg_status of this solve */
} dg_solve_info;

/* Solver for one mesh: Reynolds number Re and artificial sound speed c
 * (Eq. ns_artcomp; the paper's default c = 1e3). */
dg_status dg_solver_create(dg_mesh* mesh, double Re, double c, dg_solver** out);
void dg_solver_destroy(dg_solver* solver);

/* Solve one stage system on the solver's stream (see the stream note above):
 *   system MOMENTUM:  (co) applied per component with advecting field ubar,
 *                     rhs and x have n_dofs_u doubles (all components);
 *   system HELMHOLTZ: (alpha M^p + K), rhs and x have n_dofs_p doubles.
 * x: in the guess when opts->guess == DG_GUESS_GIVEN (ignored otherwise),
 * out the solution (best iterate on DG_ENOCONV).  Synchronous. */
dg_status dg_solve_stage(dg_solver* solver, const dg_momentum_coeffs* co, double alpha,
                         const double* ubar, const double* rhs, double* x,
                         const dg_solve_opts* opts, dg_solve_info* info);

/* TR-BDF2 step parameters.  dt, gamma (<= 0: 2 - sqrt(2)); extrapolate: 1 =
 * extrapolated advecting fields (linear to t^{n+gamma/2} from u^n and
 * u^{n-1+gamma}; linear to t^{n+1} from u^{n+gamma} and u^n), 0 = lagged
 * (u^n, u^{n+gamma}).  uD_*: Dirichlet data as velocity-layout nodal fields
 * whose wall traces are the data, or NULL (homogeneous).  Walls are
 * impermeable: the data must be tangential, u_D . n = 0 on every wall
 * (no-slip walls, moving lids).  There the Lax-Friedrichs speed of the
 * paper's boundary flux (Section 3: the mirror state 2 u_D - ubar+, speed
 * max(|ubar+ . n|, |(2 u_D - ubar+) . n|)) is |ubar+ . n|, which is what the
 * operators use; inflow and outflow data are not supported and are not
 * checked.  f_*: forcing at velocity nodes at t^n, t^{n+gamma}, t^{n+1}, or
 * NULL. */
typedef struct {
  double dt, gamma;
  int32_t extrapolate;
  const double* uD_stage1;
  const double* uD_stage2;
  const double* f_n;
  const double* f_ng;
  const double* f_n1;
  dg_solve_opts mom, helm;
  /* Fully nonlinear momentum stages (Section 2, the fixed-point alternative
   * to the linearised advecting fields, needed at larger Courant numbers):
   * fixed_point <= 1 takes one linear solve per stage with the advecting
   * field above; fixed_point = K > 1 takes at most K Picard solves, each with
   * the previous solve's velocity as advecting field (the first one starts
   * from the field above), stopping once the relative 2-norm change of the
   * iterate ||u_k - u_{k-1}|| / ||u_k|| drops below fixed_point_tol.  The
   * explicit advection term of stage 1 is then advected by u^n, as in the
   * fully implicit trapezoidal stage.  The stage's dg_solve_info sums the
   * Krylov iterations of its Picard solves (res0 of the first, res_final of
   * the last); dg_solver_get_fixed_point gives the Picard counts. */
  int32_t fixed_point;
  double fixed_point_tol;
} dg_step_params;

/* The two comparison projection schemes of Section 2 on the same DG
 * operators, in artificial compressibility form (a project addition for the
 * paper's method comparison):
 *  DG_SCHEME_BCG (Bell-Colella-Glaz, Eqs. momentum_BCG, helmholtz_BCG):
 *    (M/dt + A/(2Re) + C(w)/2) u* = M u^n/dt + E_v u^n/(2Re) + E_a(w) u^n/2
 *        + G p^n (+ data, + M (f^n + f^{n+1})/2), with the midpoint advecting
 *    field w = (u* + u^n)/2 found by Picard solves (fixed_point > 1, starting
 *    from u^n, stopping below fixed_point_tol as in trbdf2_step) or, with
 *    fixed_point <= 1, one solve with w = 3/2 u^n - 1/2 u^{n-1};
 *    (alpha M^p + K) dp = D u* / dt, alpha = 1/(c dt)^2;
 *    u^{n+1} = u* - dt M^-1 P dp, p^{n+1} = p^n + dp.
 *  DG_SCHEME_BDF2 (Guermond-Quartapelle, Eqs. momentum_HI, helmholtz_HI):
 *    (3M/(2dt) + A/Re + C(w)) u* = M (4u^n - u^{n-1})/(2dt) + G p^n
 *        (+ data, + M f^{n+1}), w the previous step's predicted velocity
 *    u^{n,*} (u^n on the solver's first such step);
 *    u** = u* + tau M^-1 P p^n, tau = 2dt/3,
 *    (alpha M^p + K) p^{n+1} = alpha M^p p^n + D u** / tau, alpha = 1/(c tau)^2,
 *    u^{n+1} = u** - tau M^-1 P p^{n+1}.
 * The solver keeps u^{n-1} as its history level (dg_solver_set_history sets
 * it; before the first step it is u^n); a solver steps with one scheme.  uD:
 * Dirichlet data at t^{n+1} (tangential, as in dg_step_params) or NULL;
 * f_n, f_n1: forcing at t^n and t^{n+1} or NULL.  info[2] (host): momentum,
 * Helmholtz.  Synchronous, on the solver's stream. */
enum { DG_SCHEME_BCG = 1, DG_SCHEME_BDF2 = 2 };

typedef struct {
  int32_t scheme;
  double dt;
  const double* uD;
  const double* f_n;
  const double* f_n1;
  dg_solve_opts mom, helm;
  int32_t fixed_point;
  double fixed_point_tol;
} dg_projection_params;

dg_status dg_projection_step(dg_solver* solver, const dg_projection_params* params, double* u,
                             double* p, dg_solve_info info[2]);

/* Picard solves taken by each momentum stage of the last trbdf2_step
 * (iterations[0] stage 1, [1] stage 2; 1 without fixed-point iterations) or
 * by the momentum predictor of the last dg_projection_step (iterations[0]). */
dg_status dg_solver_get_fixed_point(const dg_solver* solver, int32_t iterations[2]);

/* One TR-BDF2 step (Section 2, Eqs. first_stage ... helmholtz3a; algebraic
 * form of Section 3): u (n_dofs_u) in u^n, out u^{n+1}; p (n_dofs_p) in p^n,
 * out p^{n+1}.  The solver keeps u^{n-1+gamma} for the stage-1 extrapolation
 * (set with dg_solver_set_history; before the first step it is u^n).
 * info[4] (host): momentum 1, Helmholtz 1, momentum 2, Helmholtz 2. */
dg_status trbdf2_step(dg_solver* solver, const dg_step_params* params, double* u, double* p,
                      dg_solve_info info[4]);

/* Learned initial guess (a project addition; the paper starts each solve from
 * the previous level).  For each (stage, system) the solver keeps the last
 * four solutions; DG_GUESS_EXTRAP starts from their linear extrapolation
 * 2 x_{k-1} - x_{k-2} and DG_GUESS_LEARNED adds the output of a per-cell MLP
 * (4 linear layers n_in -> hidden -> hidden -> hidden -> n_out, SiLU; inputs
 * the cell's DoFs of those four solutions, as x_{k-1} and its first, second
 * and third backward differences in time, and of the right-hand side, each
 * block scaled by 1/RMS of it; output times the RMS of the second
 * difference, the size of the extrapolation error).  BF16
 * weights and activations with FP32 accumulation; the output layer starts at
 * zero, so an untrained net gives the extrapolated guess.  train = 1 takes
 * one Adam step per solve on that solve's cells (target: the converged
 * solution).  systems: bit 0 pressure Helmholtz, bit 1 momentum.  hidden and
 * seed apply when a net is first built. */
typedef struct {
  int32_t enable;
  int32_t train;
  int32_t systems;
  int32_t hidden;
  float lr;
  uint64_t seed;
} dg_guess_opts;

dg_status dg_guess_configure(dg_solver* solver, const dg_guess_opts* opts);

typedef struct {
  int64_t train_steps;   /* optimiser steps taken */
  double last_loss;      /* mean squared error of the last training batch (scaled units) */
  int32_t history[4];    /* stored solutions per slot (stage 1 momentum, stage 1 Helmholtz, stage 2 ...) */
} dg_guess_stats;

dg_status dg_guess_get_stats(const dg_solver* solver, dg_guess_stats* stats);

/* The learned guess's network on its own (gradient checks): weights packed as
 * W1 [hidden x n_in], b1, W2 [hidden x hidden], b2, W3, b3, W4 [n_out x hidden],
 * b4 (FP32, device); X [M x n_in] FP32 (rounded to BF16 on entry); hidden
 * activations rounded to BF16 after SiLU; Y [M x n_out] FP32 out.  When T is
 * not NULL: loss (host float) = mean((Y - T)^2) and grad (device, packed like
 * weights) = its gradient, with the error gradients rounded to BF16 before
 * each product.  Allocates its own scratch; synchronous. */
dg_status dg_mlp_forward_backward(int64_t M, int32_t n_in, int32_t hidden, int32_t n_out,
                                  const float* weights, const float* X, const float* T, float* Y,
                                  float* loss, float* grad, void* stream);

/* Inference of the same network (the solver's path once training stops):
 * Y = f(X), same layout and rounding points as dg_mlp_forward_backward.
 * With hidden = 128 and n_out <= 128 it runs as one fused kernel that keeps
 * the BF16 weights in shared memory (when they fit) and chains the four
 * tensor-core layers per 16-row tile; otherwise layer by layer.  Allocates
 * its own scratch; synchronous. */
dg_status dg_mlp_infer(int64_t M, int32_t n_in, int32_t hidden, int32_t n_out,
                       const float* weights, const float* X, float* Y, void* stream);

/* The caller's stream (a cudaStream_t; NULL = the legacy default stream, the
 * default): every later solver call (dg_solve_stage, trbdf2_step,
 * dg_solver_set_history) first waits for the work enqueued on it, so inputs
 * filled on a non-blocking stream (a framework's side stream, a per-thread
 * default stream) are complete before the solver reads them.  The solver
 * still computes on its own stream and synchronises it before returning. */
dg_status dg_solver_set_stream(dg_solver* solver, void* stream);

/* Set (device pointer, n_dofs_u) or clear (NULL) the stored u^{n-1+gamma}. */
dg_status dg_solver_set_history(dg_solver* solver, const double* u_hist);

/* Tracing: with on != 0, trbdf2_step records CUDA events on the solver's
 * stream at its phase boundaries and accumulates the time (ms) spent in
 * 0 extrapolation and momentum right-hand sides, 1 initial guesses (history,
 * learned prediction and training), 2 momentum solves, 3 projections,
 * pressure right-hand sides and velocity updates, 4 Helmholtz solves
 * (phase_ms[5] stays 0); set_tracing resets the totals. */
dg_status dg_solver_set_tracing(dg_solver* solver, int32_t on);
dg_status dg_solver_get_trace(const dg_solver* solver, double phase_ms[6], int64_t* steps);

/* Checkpoint / resume of the solver state (history level, learned-guess
 * weights and optimiser moments) to a host file path. */
dg_status dg_solver_save(const dg_solver* solver, const char* path);
dg_status dg_solver_load(dg_solver* solver, const char* path);

/* Pressure Helmholtz solve that allocates nothing.  The paper has no
 * counterpart: this is a service for callers that cannot allocate device
 * memory at the point of the solve (a fixed up-front memory budget, a
 * framework that owns the device heap, no dg_solver available).  Same system
 * and algorithm as dg_solve_stage with system DG_SYS_HELMHOLTZ: (alpha M^p + K)
 * x = rhs by flexible CG with precond DG_PC_JACOBI or DG_PC_NONE and guess
 * DG_GUESS_ZERO or DG_GUESS_GIVEN; rhs and x are caller-owned device arrays of
 * n_dofs_p doubles, work is enqueued on `stream` and the call synchronises it.
 * Scratch is a fixed library-owned device array (about 12.6 MB on every GPU
 * that loads the library, held until exit), so systems with more than
 * 262144 pressure DoFs are rejected with DG_EINVAL.  The first call on a
 * device looks up that array's device address; make it before any stream
 * capture.  The mesh's device must be current (DG_EINVAL otherwise).  Calls
 * share the array: calls that overlap on the GPU race and must be
 * serialised by the caller.  info (host) may be NULL. */
dg_status dg_solve_helmholtz_noalloc(dg_mesh* mesh, double alpha, const double* rhs, double* x,
                                     const dg_solve_opts* opts, dg_solve_info* info,
                                     void* stream);

/* Diagnostics (no counterpart in the paper): number of CUDA kernels this
 * library has launched in the calling process so far. */
int64_t dg_kernel_launches(void);

const char* dg_status_string(dg_status status);
const char* dg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DG_H */
