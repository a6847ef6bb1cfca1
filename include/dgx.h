/*
 * dgx.h -- C ABI of the GB300 (sm_103a) library for the pressure solve and the
 * explicit fluxes of the IMEX discontinuous-Galerkin compressible-Euler
 * scheme of Orlando, Benacchio & Bonaventura, "Improving the scalability of a
 * high-order atmospheric dynamics solver based on the deal.II library"
 * (arXiv:2505.00384).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Unknowns are nodal DG fields of degree r on the (r+1)^3 Gauss-Lobatto
 *    points of each hexahedral cell (Sec. 2).  DoF index
 *    cell * (r+1)^3 + a + (r+1) b + (r+1)^2 c (x fastest), with
 *    cell = cx + nx (cy + ny cz).  N = nx ny nz (r+1)^3.  Vector fields are
 *    three consecutive N-blocks (x, y, z components).
 *  - Every array argument is a DEVICE pointer on the context's device unless
 *    the comment says host.  Arrays are contiguous; the element type is
 *    double for DGX_F64 and float for DGX_F32.  The caller owns every array
 *    it passes; the library never frees or keeps them beyond the call except
 *    where stated (dgx_set_coefficients copies).
 *  - The library owns its workspace (geometry tables, coefficient copies,
 *    preconditioner diagonals, Krylov bases) and frees it in dgx_destroy.
 *  - Calls are enqueued on the stream given to dgx_create and return before
 *    the GPU finishes, except dgx_solve_pressure and dgx_imex_step, which
 *    return after the solve because they fill an info struct.
 *  - Return value: 0 = success, > 0 = soft status (DGX_NOT_CONVERGED), < 0 =
 *    error (nothing useful was written).  dgx_last_error gives a message.
 */
#ifndef DGX_H
#define DGX_H

#ifdef __cplusplus
extern "C" {
#endif

#define DGX_OK 0
#define DGX_NOT_CONVERGED 1
#define DGX_FALLBACK_USED 2
#define DGX_ERR_ARG (-1)
#define DGX_ERR_OOM (-2)
#define DGX_ERR_CUDA (-3)
#define DGX_ERR_BREAKDOWN (-4)
#define DGX_ERR_DEVICE_TIMEOUT (-5)
#define DGX_ERR_STATE (-6)

/* Arithmetic of an operator application. */
#define DGX_F64 0
#define DGX_F32 1

/* Jacobi preconditioners of Sec. 3.1. */
#define DGX_PC_NONE 0
#define DGX_PC_HELMHOLTZ 1       /* inverse diagonal of S~ (Helmholtz preconditioner)        */
#define DGX_PC_INTERNAL_ENERGY 2 /* inverse diagonal of D (internal-energy preconditioner)  */
#define DGX_PC_LEARNED 3         /* Helmholtz Jacobi guess plus a learned correction
                                    (dgx_learned_*); DGX_SOLVER_FGMRES only.  The FP64
                                    residual judges it: a cycle that does not halve the
                                    residual, or a non-finite direction, switches the
                                    rest of the solve to DGX_PC_HELMHOLTZ and the call
                                    returns DGX_FALLBACK_USED                           */
#define DGX_PC_MULTIGRID 4       /* one geometric-multigrid V-cycle (dgx_mg_setup first);
                                    DGX_SOLVER_CG (SPD systems, Sec. 3.1) or
                                    DGX_SOLVER_FGMRES                                     */

/* Krylov methods (Sec. 3.1: GMRES for the non-symmetric Schur system, CG
 * for the symmetric positive definite case). */
#define DGX_SOLVER_FGMRES 0 /* flexible GMRES in FP64                                         */
#define DGX_SOLVER_CG 1     /* preconditioned CG in FP64 (S must be SPD)                       */
#define DGX_SOLVER_MIXED 2  /* FP64 flexible GMRES whose preconditioner is an FP32 GMRES solve */

typedef struct dgx_ctx dgx_ctx;

/* Mesh of Sec. 3: structured hexahedra on [0,Lx] x [0,Ly] x [0,Lz],
 * terrain-following in z (z = zeta + h(x,y) (1 - zeta/Lz), zeta uniform).
 * terrain: 0 flat; 1 bell h = h_c / (1 + ((x-x_c)^2 + (y-y_c)^2)/a_c^2);
 *          2 bell of Sec. 3, h = h_c [1 + ((x-x_c)^2 + (y-y_c)^2)/a_c^2]^(-3/2).
 * bc_lateral: 0 slip walls on the four lateral faces; 1 far field (the
 * explicit flux sees the background plus (u_bar,0,0); in the pressure operator
 * the perturbation pressure takes its far-field value 0 in the B flux and the
 * enthalpy flux is transmissive); 2 periodic in x and y (the terrain must
 * match on opposite faces, e.g. a centred hill).  Bottom and top are slip
 * walls.
 * n_q: Gauss points per direction of the consistent rule; 0 selects 2r+1
 * (Sec. 3.3), the only value the GPU kernels accept.
 * refine: a non-conforming mesh (Sec. 3: neighbouring cells of different
 * resolution horizontally and vertically) when the box [refine[0], refine[1])
 * x [refine[2], refine[3]) x [refine[4], refine[5]) of base cells is not
 * empty: each base cell of the box is split 2 x 2 x 2.  Layout of every
 * per-DoF array: the nx*ny*nz base cells first (x fastest), those inside the
 * box "dead" (they hold no unknowns: inputs must be 0 there, outputs are 0
 * there), then the children as one structured block of (2 bx)(2 by)(2 bz)
 * cells, x fastest; (r+1)^3 nodes per cell as on conforming meshes.  A
 * child's map is its parent's isoparametric map restricted to the child, so
 * the faces between children and base cells (2:1 "hanging" faces) are
 * watertight; their face terms are integrated with the children's face rule
 * on both sides (conservative).  The box must leave at least one base cell
 * outside it and, with periodic lateral faces, stay clear of them.  On
 * non-conforming meshes the operator, its parts, the diagonals, the FP64, CG
 * and mixed solvers with the Jacobi preconditioners, node coordinates,
 * background, explicit tendencies and the IMEX step are available (the step
 * sets the dead cells of the state to the background at rest: rho = rho_bar,
 * u = 0, p = p_bar); the learned and multigrid preconditioners, the consistent
 * mass rule, ensembles and dgx_apply_operator_noalloc return DGX_ERR_STATE. */
typedef struct {
  int nx, ny, nz;
  int degree;
  int n_q;
  int terrain;
  int bc_lateral;
  int reserved;
  double Lx, Ly, Lz;
  double h_c, a_c, x_c, y_c;
  int refine[6];
} dgx_mesh_desc;

/* Hydrostatic background (Sec. 3): kind 0 isothermal at T (p = p0 exp(-g z/(R T))),
 * kind 1 the constant-buoyancy-frequency state of Sec. 3 with N_bv, T = T_ref
 * (rho = rho_ref (p/p0)^(1/gamma) exp(-N^2 z/g), p from hydrostatic balance:
 * p = p0 {1 - (g^2/N^2) Gamma rho_ref/p0 [1 - exp(-N^2 z/g)]}^(1/Gamma)). */
typedef struct {
  int kind;
  int reserved;
  double T, p0, N_bv, R, gamma, g, u_bar;
} dgx_background;

typedef struct {
  int method;        /* DGX_SOLVER_*                                                     */
  int pc;            /* DGX_PC_* (right preconditioning)                                 */
  int restart;       /* FGMRES restart length m (<= 64)                                  */
  int maxit;         /* maximum outer iterations                                         */
  double tol;        /* relative residual ||b - S x||_2 / ||b||_2 checked in FP64        */
  int inner_restart; /* DGX_SOLVER_MIXED: FP32 GMRES restart length                      */
  int inner_maxit;   /* DGX_SOLVER_MIXED: FP32 iterations per outer iteration            */
  double inner_tol;  /* DGX_SOLVER_MIXED: relative tolerance of the FP32 inner solve      */
  int use_x0;        /* 1: x holds the initial guess; 0: start from zero                  */
  int reserved;
} dgx_solve_opts;

typedef struct {
  int status;          /* DGX_OK, DGX_NOT_CONVERGED or DGX_FALLBACK_USED                  */
  int iterations;      /* outer (FP64) Krylov iterations                                 */
  int inner_iterations;/* FP32 iterations (DGX_SOLVER_MIXED)                             */
  int operator_f64;    /* FP64 operator applications, all that ran (on meshes up to 2^20
                          unknowns, FGMRES applies the operator to the next direction
                          while the host reads the Arnoldi scalars: one extra
                          application at the end of each cycle)                          */
  int operator_f32;    /* FP32 operator applications of the inner iterations (one each;
                          the inner solve's speculative last one is not counted)         */
  int fallback;        /* DGX_PC_LEARNED: 1 if the solve switched to the Helmholtz Jacobi */
  double relres;       /* final relative residual ||b - S x|| / ||b|| in FP64 (see below)  */
  double seconds;      /* wall time of the call                                          */
} dgx_solve_info;

/* Create a context on CUDA device `device`, enqueueing all work on
 * `cuda_stream` (a cudaStream_t; NULL = legacy default stream). */
int dgx_create(dgx_ctx **ctx, int device, void *cuda_stream);
void dgx_destroy(dgx_ctx *ctx);
const char *dgx_last_error(const dgx_ctx *ctx);

/* Build the mesh and its geometry tables (per-column terrain heights and
 * their derivatives at the quadrature points), Sec. 2-3.  Replaces any
 * earlier mesh and drops coefficients and diagonals. */
int dgx_mesh_build(dgx_ctx *ctx, const dgx_mesh_desc *desc);
/* N, the number of pressure DoFs; -1 without a mesh. */
long long dgx_num_dofs(const dgx_ctx *ctx);
/* Physical coordinates of all DoF nodes: X (device, 3N doubles). */
int dgx_node_coords(dgx_ctx *ctx, double *X);

/* Background state (Sec. 3); needed by the IMEX step. */
int dgx_set_background(dgx_ctx *ctx, const dgx_background *bg);
/* Nodal background density and pressure (device, N doubles each). */
int dgx_background_fields(dgx_ctx *ctx, double *rho_bar, double *p_bar);

/* Coefficients of the Schur operator of one fixed-point iteration (Sec. 2):
 * rho_l = rho^(l) (nodal, N doubles), p_k = total pressure of the previous
 * fixed-point iterate (nodal, N doubles), a_dt = a~_ll * dt, gamma.  The
 * library copies both fields (FP64 and FP32 copies) and the coefficient
 * factor a_dt gamma/(gamma-1) p_k at the Gauss points; the Helmholtz and
 * internal-energy diagonals (Sec. 3.1) follow on first use (FP64, or FP32
 * when only the mixed solver's FP32 inner solve needs them). */
int dgx_set_coefficients(dgx_ctx *ctx, const double *rho_l, const double *p_k, double a_dt, double gamma);

/* Quadrature of the density-weighted mass A(rho) (Sec. 3.3), a setting of
 * the context that holds for every application or inversion of A in it: the
 * operator S (both precisions), dgx_apply_grad, dgx_apply_mass_inverse,
 * dgx_apply_mass and dgx_imex_step.  The ensemble solver and
 * dgx_apply_operator_noalloc always use the fast rule.
 *   DGX_MASS_FAST        r+1 Gauss points per direction, inverted in closed form
 *                        by the fast inverse S^-T J^-1 S^-1 (the default).
 *   DGX_MASS_CONSISTENT  the consistent 2r+1 point rule of the other integrals;
 *                        A^-1 by preconditioned conjugate gradients inside each
 *                        cell, preconditioned by the fast inverse, to relative
 *                        residual cg_tol (FP32: at least 1e-5) within cg_maxit
 *                        iterations.
 * Errors: DGX_ERR_ARG for an unknown rule, cg_tol <= 0 or cg_maxit < 1. */
#define DGX_MASS_FAST 0
#define DGX_MASS_CONSISTENT 1
int dgx_set_mass_rule(dgx_ctx *ctx, int rule, double cg_tol, int cg_maxit);
/* Statistics of the consistent-mass conjugate gradients since the previous
 * call (synchronises the context's stream, then resets them): the largest
 * iteration count of any cell solve and the number of cell solves that
 * stopped at cg_maxit or met a non-finite residual. */
int dgx_mass_cg_stats(dgx_ctx *ctx, int *max_iterations, int *unconverged);

/* y = S x = D x - C A^-1 B x, the matrix-free Schur operator of the
 * fixed-point equation of Sec. 2 with the block-diagonal inverse of Sec. 3.3
 * (the fast inverse, or the consistent mass's, per dgx_set_mass_rule);
 * x, y: N elements of type `prec`.  x and y must not alias. */
int dgx_apply_operator(dgx_ctx *ctx, int prec, const void *x, void *y);
/* V = A^-1 B p (the pressure-gradient step, 3N out) and y = D p - C V
 * (the divergence step, N out): the two halves of dgx_apply_operator. */
int dgx_apply_grad(dgx_ctx *ctx, int prec, const void *p, void *V);
int dgx_apply_div(dgx_ctx *ctx, int prec, const void *V, const void *p, void *y);
/* out = A_rho^-1 in (3N -> 3N): the fast inverse S^-T J^-1 S^-1 of Sec. 3.3,
 * or the consistent mass's inverse (dgx_set_mass_rule). */
int dgx_apply_mass_inverse(dgx_ctx *ctx, int prec, const void *in, void *out);
/* y = P^-1 x for the Jacobi preconditioner `pc` (Sec. 3.1). */
int dgx_apply_preconditioner(dgx_ctx *ctx, int pc, int prec, const void *x, void *y);
/* The (non-inverted) diagonal of `pc` (FP64, N doubles). */
int dgx_preconditioner_diagonal(dgx_ctx *ctx, int pc, double *d);

/* Solve S x = b (Sec. 3.1) to ||b - S x|| <= tol ||b|| in FP64.  b, x:
 * device, N doubles.  FGMRES computes b - S x0 with an FP64 application when
 * a solve starts (b itself when use_x0 = 0) and, after each restart cycle, as
 * r0 - sum_j y_j (S z_j) from the FP64 products of that cycle (S is linear).
 * Returns DGX_OK, DGX_NOT_CONVERGED (x holds the last iterate),
 * DGX_FALLBACK_USED (DGX_PC_LEARNED only) or an error (DGX_ERR_BREAKDOWN on a
 * NaN or zero Krylov scalar). */
int dgx_solve_pressure(dgx_ctx *ctx, const double *b, double *x, const dgx_solve_opts *opts,
                       dgx_solve_info *info);

/* Default options: FGMRES(30), Helmholtz preconditioner, tol 1e-8. */
void dgx_default_solve_opts(dgx_solve_opts *opts);

/* ---------------------------------------------------------------- IMEX step
 * The IMEX Runge-Kutta stage equations of Sec. 2 (companion tableaux A, A~).
 * State: rho (N), u (3N), p (N) nodal fields, total (not perturbation)
 * values, FP64 device arrays.  Stage l: rho^(l) from the explicit continuity
 * sums; momentum and energy coupled through the pressure (Helmholtz) equation,
 * solved by K fixed-point iterations, each one linear solve S p' = G - C A^-1 F
 * for p' = p - p_bar (background subtracted in FP64), then
 * U = A^-1 (F - B p').  Explicit terms: advective fluxes of rho, rho u, rho k
 * (local Lax-Friedrichs flux) and the gravity work rho g.u; implicit terms: the
 * pressure gradient with buoyancy rho' g and the enthalpy flux.  Bottom and
 * top slip walls; lateral faces per dgx_mesh_desc.bc_lateral (far field:
 * background density and (u_bar, 0, 0)). */

/* Tableaux (host, s x s row-major, 2 <= s <= 4): A strictly lower, A~ lower
 * with an explicit first stage (A~ first row zero) and a~_ll > 0 for l > 1.
 * The new state is the last stage (stiffly accurate pairs such as
 * ARS(2,2,2)).  dt > 0; K fixed-point iterations per implicit stage. */
int dgx_set_imex(dgx_ctx *ctx, int s, const double *A, const double *At, double dt, int K);

/* Explicit tendencies of (rho, u) as dual vectors (tested against each basis
 * function): Erho (N) = weak -div(rho u), Em (3N) = weak -div(rho u_d u),
 * Ee (N) = weak -div(rho k u) + int rho g.u psi.  Needs the background. */
int dgx_explicit_tendencies(dgx_ctx *ctx, const double *rho, const double *u, double *Erho, double *Em, double *Ee);
/* out = A(rho) in (3N -> 3N): the density-weighted mass of Sec. 3.3 applied
 * forward, with the context's quadrature (dgx_set_mass_rule). */
int dgx_apply_mass(dgx_ctx *ctx, const double *rho, const double *in, double *out);
/* out_i = int rho |u|^2/2 psi_i (N), consistent rule. */
int dgx_kinetic_mass(dgx_ctx *ctx, const double *rho, const double *u, double *out);

typedef struct {
  int steps;             /* steps completed                                              */
  int solves;            /* pressure solves (stages x fixed-point iterations x steps)     */
  int krylov_iterations; /* outer Krylov iterations, all solves                          */
  int inner_iterations;  /* FP32 iterations (DGX_SOLVER_MIXED)                           */
  int operator_f64;
  int operator_f32;
  int status;            /* DGX_OK, or DGX_NOT_CONVERGED if any solve stopped at maxit   */
  int reserved;
  double max_relres;     /* largest final relative residual of the solves                */
  double seconds;        /* wall time of the call                                        */
  double seconds_solve;  /* of which inside dgx_solve_pressure                           */
} dgx_step_info;

/* Advance (rho, u, p) in place by nsteps IMEX steps.  opts: the pressure
 * solves (NULL: defaults; the initial guess is always the previous iterate).
 * Needs mesh, background and tableau.  Returns after the last step; DGX_OK,
 * DGX_NOT_CONVERGED or an error.  Workspace (9 N s + 27 N doubles) is owned by
 * the context. */
int dgx_imex_step(dgx_ctx *ctx, double *rho, double *u, double *p, int nsteps, const dgx_solve_opts *opts,
                  dgx_step_info *info);

/* Recorder of the pressure systems dgx_imex_step solves.  From this call on,
 * every `stride`-th solve (the stride-th, 2 stride-th, ...; counting all
 * stages and fixed-point iterations) appends one record of 4 N + 2 doubles to
 * `store` (device, caller-owned, capacity records): rho^(l), p_k (the
 * coefficients of dgx_set_coefficients), the right-hand side b, the solution
 * x (p' of Sec. 2 after the solve), then a~_ll dt and gamma.  Recording stops
 * when `capacity` records are written; store = NULL or capacity = 0 turns it
 * off.  dgx_imex_recorded gives the number written so far. */
int dgx_imex_record(dgx_ctx *ctx, double *store, int capacity, int stride);
int dgx_imex_recorded(const dgx_ctx *ctx);

/* ------------------------------------------------------- learned preconditioner
 * The paper preconditions the Schur system with a Jacobi diagonal (Sec. 3.1);
 * this extension adds a learned correction that flexible GMRES accepts as a
 * variable preconditioner:  z = M(v) = j + s c,  j = D_H^-1 v (the Helmholtz
 * Jacobi guess of the current coefficients), s = sqrt(mean(j^2)), and c the
 * output of a network of `layers` 3x3x3 convolutions (zero padding, ReLU
 * between layers, `channels` hidden channels) applied to the cell-DoF tensor:
 * the N nodal values laid out as a grid of (nz n) x (ny n) x (nx n) points,
 * n = r+1, each cell's n^3 nodes in their own block (grid index
 * gx + X (gy + Y gz), X = nx n, Y = ny n).  Input channels, per grid point:
 *   0  j / s                         1  log(d_i / mean(d)), d the Helmholtz diagonal
 *   2  p_k / mean(p_k) - 1           3  rho / mean(rho) - 1
 *   4  h(x, y) / Lz (terrain height at the node's column)
 * Weights are stored in bfloat16 (FP32 master copies for training), biases
 * in FP32; every convolution accumulates in FP32.  Parameter vector layout
 * (FP32): for each layer, W[co][ci][kz][ky][kx] then b[co].
 * Training pairs (v, e) with S e = v are stored in normalised form: the five
 * channels and the target t = e / s; the loss of a batch of B pairs is
 *   L = (1/B) sum_b || ch0_b + c_b - t_b ||^2 / || t_b ||^2
 * (equal to ||M(v) - e||^2 / ||e||^2 per pair), minimised by Adam.  The
 * network and the samples survive dgx_mesh_build while the grid extents
 * X, Y, Z stay the same (another terrain, say); other extents drop the
 * samples.  All arrays device unless stated. */
typedef struct {
  int epochs;              /* passes over the training samples                     */
  int batch;               /* pairs per Adam step (1..256)                          */
  double lr, lr_final;     /* learning rate, cosine-decayed from lr to lr_final    */
  double beta1, beta2, eps;/* Adam                                                 */
  unsigned long long seed; /* shuffling of the training samples                    */
  int shuffle;             /* 0: samples in insertion order                        */
  int reserved;
} dgx_train_opts;

typedef struct {
  int steps;               /* Adam steps taken                                     */
  int train_samples, test_samples, reserved;
  double loss_train0, loss_test0; /* before training (mean over the samples)       */
  double loss_train, loss_test;   /* after training                                */
  double seconds;
} dgx_train_info;

/* Create (or replace) the network: 2 <= layers <= 16, channels a multiple of
 * 8 in 8..64; He-normal weights from `seed` (splitmix64 + Box-Muller), the
 * last layer zero so that M starts as the Jacobi preconditioner. */
int dgx_learned_create(dgx_ctx *ctx, int layers, int channels, unsigned long long seed);
long long dgx_learned_num_params(const dgx_ctx *ctx);
/* FP32 parameter vector (host), layout above; set rounds weights to bfloat16
 * for use and keeps the FP32 values as master copies; resets Adam. */
int dgx_learned_get_params(dgx_ctx *ctx, float *host_params);
int dgx_learned_set_params(dgx_ctx *ctx, const float *host_params);
/* z = M(v) for the current coefficients (prec DGX_F64 or DGX_F32). */
int dgx_learned_apply(dgx_ctx *ctx, int prec, const void *v, void *z);
/* Add training pairs from one pressure system: sets the coefficients
 * (as dgx_set_coefficients), stores (b, x) and then, from restarted FGMRES
 * cycles of `stride` Jacobi iterations from x = 0, the pairs (r_k, x - x_k)
 * (residual and error of the k-th cycle) while ||r_k|| >= 1e-6 ||b||, up to
 * `pairs` pairs in all.  x must solve S x = b to ~1e-10.  test != 0 keeps the
 * pairs out of training (held out for dgx_train_info.loss_test). */
int dgx_learned_add_system(dgx_ctx *ctx, const double *rho, const double *pk, double a_dt, double gamma,
                           const double *b, const double *x, int pairs, int stride, int test);
int dgx_learned_num_samples(const dgx_ctx *ctx, int *train, int *test);
/* Sample i (insertion order) as 6 G floats (host): channels 0..4 then t. */
int dgx_learned_sample(dgx_ctx *ctx, int i, float *host_out);
int dgx_learned_clear_samples(dgx_ctx *ctx);
/* Mean loss over samples first..first+count-1 (one batch, count <= 256) and
 * its gradient w.r.t. the parameter vector (host FP32, may be NULL); no update. */
int dgx_learned_loss(dgx_ctx *ctx, int first, int count, double *loss, float *grad_host);
/* Train on the non-test samples with Adam; fills info (may be NULL). */
int dgx_learned_train(dgx_ctx *ctx, const dgx_train_opts *opts, dgx_train_info *info);
void dgx_default_train_opts(dgx_train_opts *opts);

/* Allocation-free variant of dgx_apply_operator.  The paper has no
 * counterpart: this serves callers that cannot allocate device memory when
 * they apply the operator (an application whose pool allocator owns all
 * device memory after start-up, or a time-critical loop that must not call
 * cudaMalloc).  y = S x exactly as dgx_apply_operator (same kernels, same
 * result), but the intermediate V = A^-1 B x (3N elements of type `prec`)
 * lives in a fixed file-scope device array of DGX_NOALLOC_SCRATCH_BYTES
 * (16 MiB) that every GPU loading the library holds until process exit; the
 * call allocates nothing.  Limit: 3 N sizeof(prec) <= 16 MiB, i.e.
 * N <= 699050 in FP64 and N <= 1398101 in FP32; larger meshes get
 * DGX_ERR_ARG with a message.  The first call on a device looks up the
 * array's device address with that device current; make that first call
 * before any stream capture.  The address is kept for the life of the
 * process: a cudaDeviceReset (or anything else that unloads the library's
 * module from the device) between calls makes the entry point unusable.  All calls share the one array and it keeps the
 * last call's contents: calls whose GPU work overlaps (other streams or
 * contexts on the same device) race on it and must be serialised by the
 * caller.  Nothing needs clearing: each call writes all 3N entries it reads.
 * Errors as dgx_apply_operator. */
#define DGX_NOALLOC_SCRATCH_BYTES (16u << 20)
int dgx_apply_operator_noalloc(dgx_ctx *ctx, int prec, const void *x, void *y);

/* Arithmetic of the explicit side of the step: the explicit fluxes
 * (dgx_explicit_tendencies) and the consistent-rule mass terms of the stage
 * right-hand sides (dgx_kinetic_mass and the IMEX step's rho' g and kinetic
 * terms): 1 (default) double-words on the FP32 pipes (hi + lo float pairs,
 * compensated line products, about 48 bits; degrees up to 4, higher degrees
 * use the FP64 pipe), 0 the FP64 pipe.  Both agree with the FP64 oracle to
 * 1e-12.  DGX_ERR_ARG for another value. */
int dgx_set_explicit_variant(dgx_ctx *ctx, int variant);
int dgx_explicit_variant(const dgx_ctx *ctx);

/* Algorithmic work of one dgx_apply_operator call for the current mesh (host
 * pointers, any may be NULL): floating-point operations of the implemented
 * (even-odd) sum-factorisation sweeps and pointwise work of the gradient
 * kernel (V = A^-1 B p) and of the divergence kernel (y = D p - C V), and the
 * HBM floor of the whole
 * application in bytes (p, rho, p_k read once, y written once: 32 bytes per
 * DoF in FP64). */
int dgx_operator_cost(const dgx_ctx *ctx, double *flops_grad, double *flops_div, double *bytes_f64);

/* Launch variants of the operator kernels (the two halves V = A^-1 B p and
 * y = D p - C V), all computing the same operator to rounding:
 *   0, 1, 2  one cell per CTA, one thread per 1D line of each sum-factorisation
 *            sweep, 128 / 192 / 256 threads per CTA;
 *   3, 4     fused kernels with C cells per CTA, C = 1 / 2 (degree >= 3) or
 *            4 / 8 (degree <= 2), and 32 ceil(C (2r+1)^2 / 32) threads;
 *   5, 6     (FP64 only) the fused kernels of 3, 4 computing in double-word
 *            arithmetic (pairs of FP32 numbers, about 48 significant bits,
 *            error-free transforms of Dekker, Knuth and Joldes-Muller-Popescu)
 *            on the FP64 arrays: the FP32 pipes instead of the FP64 pipe.
 * The fused kernels keep the last interpolation direction, the pointwise flux
 * and the first test direction in registers and deal the lines of several
 * cells to one CTA; a fused variant is available when its shared memory
 * (cells per CTA x per-cell plan) fits in 227 KB.  A timing autotuner picks
 * the fastest available variant before the first application on meshes of
 * 2048 cells or more (outside stream capture); smaller meshes use the
 * degree's default (-1).  dgx_mesh_build resets the choice. */
#define DGX_OP_VARIANTS 7
/* The variant in use for prec (-1: the default, not tuned; -2: bad argument). */
int dgx_operator_variant(const dgx_ctx *ctx, int prec);
/* Pin variant 0..6 for prec on the current mesh (the autotuner then leaves prec
 * alone), or hand the choice back to the autotuner with -1.  DGX_ERR_ARG for a
 * variant that is unknown or does not fit; DGX_ERR_STATE without a mesh. */
int dgx_set_operator_variant(dgx_ctx *ctx, int prec, int variant);
/* Threads per CTA of the variant in use (0 while it is the default). */
int dgx_operator_threads(const dgx_ctx *ctx, int prec);

/* Number of CUDA kernels this library has launched in this process (all
 * contexts); a diagnostic counter for benchmarks. */
long long dgx_kernel_launches(void);

/* The 1D tables every kernel of degree `degree` (1..6) works from, as built
 * on the host: N = degree+1 Gauss-Lobatto-Legendre nodes carry the nodal
 * basis (Sec. 2), Q = 2 degree + 1 Gauss points the consistent integrals, and
 * N Gauss points the fast inverse (Sec. 3.3).  Layout, row-major, x in [0, 1]:
 *   I [Q][N] l_a(g_q)     D [Q][N] l_a'(g_q)    IT, DT [N][Q] their transposes
 *   Ia [N][N] l_a(ga_q)   P [N][N] Ia^-1 [a][q]  PT [N][N] its transpose
 *   IIT, DDT, IDT [N][Q]  l_a^2, l_a'^2, l_a l_a' at g_q
 *   wq [Q], wa [N], gq [Q]  Gauss weights, fast-rule weights, Gauss points
 * Writes min(capacity, size) doubles to out (out may be NULL) and returns
 * size = 7QN + 3N^2 + 2Q + N; DGX_ERR_ARG for an unsupported degree.  Host
 * only: needs no context and no GPU. */
int dgx_basis_tables(int degree, double *out, int capacity);

/* ------------------------------------------------------ geometric multigrid
 * Sec. 3.1 solves the SPD systems with CG preconditioned by geometric
 * multigrid (and notes that no theory covers multigrid for the non-symmetric
 * Schur system, where it is an experiment here).  Hierarchy: level 0 is the
 * context's mesh and coefficients, level l halves nx, ny, nz l times (same
 * domain, degree, terrain, boundaries), so a coarse cell is 2 x 2 x 2 fine
 * cells.  Transfers: prolongation = the coarse cell's polynomial at the fine
 * GLL nodes of its children; restriction = its transpose; coarse rho, p_k = the
 * fine fields at the coarse nodes (the child holding the node, the lower one
 * at an interface).  Each level applies its own S (rediscretisation) and
 * Helmholtz Jacobi diagonal D.  Smoother: `degree` steps of Chebyshev
 * iteration on D^-1 S (Saad, Alg. 12.1) over [lambda_max / smooth_range,
 * 1.1 lambda_max], lambda_max by `power_its` power steps on D^-1 S from the
 * fixed vector v_i = frac(0.6180339887498949 (i + 1)) - 1/2.  Coarsest level:
 * CG (coarse_solver 0, SPD) or FGMRES (1) with the Helmholtz Jacobi to
 * coarse_tol within coarse_maxit iterations.  V-cycle from zero: pre-smooth,
 * restrict the residual, one cycle on the next level, prolong and correct,
 * post-smooth. */
typedef struct {
  int levels;        /* 2..12; nx, ny, nz divisible by 2^(levels-1)                 */
  int degree;        /* Chebyshev steps per smoothing (>= 1)                         */
  int power_its;     /* power iterations for lambda_max per level (>= 1)            */
  int coarse_maxit;  /* iteration bound of the coarsest solve (>= 1)                */
  int coarse_solver; /* 0: CG (SPD systems), 1: FGMRES                             */
  int reserved;
  double smooth_range; /* lambda_max / lambda_min of the smoother (> 1)             */
  double coarse_tol;   /* relative residual of the coarsest solve (> 0)             */
} dgx_mg_opts;
void dgx_default_mg_opts(dgx_mg_opts *opts); /* 3 levels, degree 3, 15 power its, 500, CG, 15, 1e-10 */
/* Build the hierarchy for the context's current mesh and coefficients
 * (allocates the coarse levels; later dgx_set_coefficients calls are picked
 * up by the next V-cycle, which restricts the new coefficients and re-estimates
 * the bounds).  dgx_mesh_build and dgx_destroy release it.  Errors: DGX_ERR_ARG
 * (options, divisibility), DGX_ERR_STATE (no mesh / coefficients). */
int dgx_mg_setup(dgx_ctx *ctx, const dgx_mg_opts *opts);
/* z = one V-cycle applied to r (device FP64, N each, distinct). */
int dgx_mg_vcycle(dgx_ctx *ctx, const double *r, double *z);
/* Number of levels and the lambda_max estimate of each (host, capacity entries). */
int dgx_mg_levels(dgx_ctx *ctx, int *levels, double *lambda_max, int capacity);

/* ---------------------------------------------------------------- ensembles
 * Several independent meshes (sizes, degrees, terrain) whose pressure
 * systems S_m p_m = b_m (Sec. 2, Sec. 3.1) are solved together.  Vectors are
 * the members' DoF blocks concatenated in member order (member m starts at
 * dgx_ensemble_offset(e, m)); all arrays are device FP64 unless stated.
 * The operator of all members of one degree runs as one kernel pair; the
 * solver is FP64 iterative refinement around an FP32 GMRES(inner_maxit)
 * cycle with the Helmholtz Jacobi preconditioner (per-member Hessenberg and
 * Givens rotations on the device).  A whole solve is one CUDA-graph launch: the
 * refinement loop is a WHILE conditional node whose condition a device kernel
 * sets from the members' FP64 residuals (bounded by maxit cycles); the host
 * reads the per-member results once.  The tile shape of the multi-mesh
 * operator (one cell per CTA at 128 / 192 / 256 threads, or the fused kernels
 * with one or more cells per CTA, in FP64 computing in double-words) is chosen
 * per degree group and precision by a timing autotuner before the graph is
 * captured. */
typedef struct dgx_ensemble dgx_ensemble;
int dgx_ensemble_create(dgx_ensemble **e, int device, void *cuda_stream, int n_members, const dgx_mesh_desc *descs);
void dgx_ensemble_destroy(dgx_ensemble *e);
const char *dgx_ensemble_last_error(const dgx_ensemble *e);
/* DoFs of member m (m = -1: total) and offset of member m in the concatenated vectors. */
long long dgx_ensemble_num_dofs(const dgx_ensemble *e, int m);
long long dgx_ensemble_offset(const dgx_ensemble *e, int m);
/* The member's own context (owned by the ensemble; for set-up calls such as
 * dgx_set_background / dgx_node_coords on that member).  Its calls run on the
 * ensemble's own stream: synchronise before reading their results on
 * another stream. */
int dgx_ensemble_member(dgx_ensemble *e, int m, dgx_ctx **ctx);
/* Concatenated rho^(l), p_k of all members; same a~_ll dt and gamma for all. */
int dgx_ensemble_set_coefficients(dgx_ensemble *e, const double *rho_all, const double *p_k_all, double a_dt,
                                  double gamma);
/* y = S x for every member (prec: DGX_F64 or DGX_F32). */
int dgx_ensemble_apply_operator(dgx_ensemble *e, int prec, const void *x_all, void *y_all);
/* Choose the tile shape of the multi-mesh operator per degree group (also done by the first solve). */
int dgx_ensemble_autotune(dgx_ensemble *e);
/* The autotuner's choice for degree group g (host outputs, any may be NULL):
 * threads per CTA in FP64 and FP32; and, for precision prec, the kernels
 * (fused = 1: the fused kernels, in FP64 computing in double-words; 0: one cell
 * per CTA) with their cells per CTA. */
int dgx_ensemble_tuning(const dgx_ensemble *e, int g, int *degree, int *members, int *threads64, int *threads32);
int dgx_ensemble_tile(const dgx_ensemble *e, int g, int prec, int *fused, int *cells_per_cta);
/* Solve all members to ||b_m - S_m x_m|| <= tol ||b_m|| (FP64).  opts: tol, maxit
 * (refinement sweeps), inner_maxit (FP32 GMRES cycle length, <= 64), inner_tol,
 * use_x0.  info: array of n_members entries (host).  Returns DGX_OK,
 * DGX_NOT_CONVERGED or an error. */
int dgx_ensemble_solve(dgx_ensemble *e, const double *b_all, double *x_all, const dgx_solve_opts *opts,
                       dgx_solve_info *info);

#ifdef __cplusplus
}
#endif
#endif
