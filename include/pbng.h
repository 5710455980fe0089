/*
 * pbng.h — C ABI of the GB300 (sm_103a) Position-Based Nonlinear Gauss-Seidel
 * library (Chen, Han, Chen, Teran, "Position-Based Nonlinear Gauss-Seidel for
 * Quasistatic Hyperelasticity", arXiv 2306.09021).
 *
 * The library solves the discrete quasistatic equilibrium of Section
 * "Discretization" (Eq. fem_qs / Eq. fem_d) for P1 tetrahedral meshes with the
 * fixed-corotated energy of Section "Constitutive Models" (Eq. cor), weak
 * constraints of Section "Weak Constraints" (zero-rest-length springs to fixed
 * targets, frictionless plane contact with k_tau = 0) and a constant body
 * acceleration.  One sweep updates every free vertex once, colour by colour
 * (Section "Coloring and Parallelism"), with the one-step modified-Newton node
 * update of Eq. pbgn_update / Eq. pbgn_dx and the SPD nodal Hessian of
 * Eq. mod_hess; Chebyshev or SOR acceleration (Section "Acceleration
 * Techniques") is applied after each whole sweep.
 *
 * General rules for every entry point:
 *  - No function aborts, throws or prints.  Each returns a pbng_status; the
 *    text of the last failure of a handle is available from pbng_last_error.
 *  - Host arrays passed in are copied; the caller keeps ownership.
 *  - Device arrays ("_dev") are owned by the caller, must be 4-byte aligned,
 *    contiguous and on the handle's device, and must stay valid until the
 *    call returns.  All GPU work is enqueued on the handle's stream.
 *  - A handle is not thread-safe.  After PBNG_ECUDA the handle must only be
 *    destroyed.
 *  - Vertex ids are 0-based int32 in the caller's order; the library keeps
 *    its own colour-ordered layout internally and translates at the boundary.
 *  - Displacements u = x - X are float32 [nv][3], row-major, in the caller's
 *    vertex order.
 */
#ifndef PBNG_H
#define PBNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PBNG_OK = 0,
    PBNG_EINVAL = 1,          /* bad argument, size or index                  */
    PBNG_ENOMEM = 2,          /* host or device allocation failed             */
    PBNG_ECUDA = 3,           /* a CUDA runtime call failed                   */
    PBNG_EDEGENERATE = 4,     /* rest tet of (near) zero volume, or a nodal
                                 Hessian that is not positive definite         */
    PBNG_EDIVERGED = 5,       /* non-finite value, residual > 1e3 r_0, or
                                 sustained growth (pbng_solve)                 */
    PBNG_ETIMEOUT = 6,        /* a bounded device wait gave up                 */
    PBNG_ENOTCONVERGED = 7    /* max_sweeps reached before rel_tol             */
} pbng_status;

typedef struct pbng_mesh pbng_mesh;   /* opaque, library-owned */

/* Acceleration of the sweeps (pbng_params.accel).  PBNG_ACCEL_CG is taken
 * by pbng_adjoint only (conjugate gradients preconditioned by the symmetric
 * block Gauss-Seidel sweep, see there); every other entry point rejects it
 * with PBNG_EINVAL. */
enum { PBNG_ACCEL_NONE = 0, PBNG_ACCEL_CHEBYSHEV = 1, PBNG_ACCEL_SOR = 2, PBNG_ACCEL_CG = 3 };
/* Precision of the sweep (pbng_params.precision).
 *   PBNG_PREC_FP32         iterate and element arithmetic float32
 *   PBNG_PREC_COMPENSATED  iterate as a float32 pair (hi + lo), element
 *                          arithmetic float32
 *   PBNG_PREC_EXTENDED     iterate as a float32 pair; every element force of
 *                          the colour passes and residuals in float-float
 *                          arithmetic (pairs of float32, about 48 bits) from
 *                          float-pair element constants, each vertex's sum in
 *                          FP64; the nodal Hessian stays float32.  Needed where
 *                          the per-element forces are far larger than their
 *                          sum: on a 64^3 cube under gravity float32 forces
 *                          and constants leave a relative-residual floor of
 *                          about 3e-4.  Ring layout only (kernel_path 0).
 *   PBNG_PREC_AUTO         colour passes and pbng_solve's residual checks as
 *                          COMPENSATED until the checks stall below 1e-2
 *                          (the best of the last 20 not below half the best
 *                          before them: the float32 passes' floor), then
 *                          EXTENDED; a float32 check that puts a component
 *                          at the tolerance is confirmed with the extended
 *                          residual first, and once half of the active
 *                          components have failed such a confirmation the
 *                          passes go EXTENDED too.  r_0 and the residuals
 *                          that pbng_sweep and
 *                          pbng_sweep_host report are extended.  Ring layout
 *                          only.
 * Every residual sums each vertex's element terms and its vertex terms in
 * float-float arithmetic and the squares in FP64 (a float32-pair sum keeps
 * FP64's accuracy here at float32 throughput: FP64 arithmetic on this GPU
 * runs at a small fraction of the float32 rate). */
enum { PBNG_PREC_FP32 = 0, PBNG_PREC_COMPENSATED = 1, PBNG_PREC_EXTENDED = 2, PBNG_PREC_AUTO = 3 };
/* Constitutive models (Section "Constitutive Models"), mu and lambda from
 * Eq. lame:
 *   PBNG_MODEL_COROTATED   Eq. cor, mu |F - R|^2 + (lambda/2)(J - 1)^2
 *   PBNG_MODEL_NEOHOOKEAN  Eq. nh, (mu/2)|F|^2 + (lambda_hat/2)(J - 1 - mu/lambda_hat)^2,
 *                          lambda_hat = mu + lambda
 *   PBNG_MODEL_STABLE_NEOHOOKEAN  Eq. snh read with lambda' on its volume
 *                          term: (mu'/2)(|F|^2 - 3) + (lambda'/2)(J - alpha)^2
 *                          - (mu'/2) log(1 + |F|^2), alpha = 1 + 3mu'/(4lambda'),
 *                          mu' = 4mu/3, lambda' = lambda + 5mu/6, so that its
 *                          Hessian at F = I is linear elasticity's (Section
 *                          "Lame Coefficients"). */
enum { PBNG_MODEL_COROTATED = 0, PBNG_MODEL_NEOHOOKEAN = 1, PBNG_MODEL_STABLE_NEOHOOKEAN = 2 };

typedef struct {
    int32_t model;          /* PBNG_MODEL_*: the energy density of Section
                               "Constitutive Models".  The nodal Hessian is
                               Eq. mod_hess_dens for every model.  The handle
                               keeps the model of its last sweep / solve /
                               autotune; pbng_residual uses it.  pbng_adjoint,
                               pbng_force, pbng_hessian_apply and
                               pbng_newton_cg use the true Hessian of the model. */
    int32_t accel;          /* PBNG_ACCEL_*                                        */
    double omega;           /* SOR weight (Section "Acceleration Techniques": 1.7) */
    double rho;             /* Chebyshev spectral estimate (0.95).  rho <= 0 with
                               PBNG_ACCEL_CHEBYSHEV: pbng_solve estimates it from
                               its FP64 residual checks (pbng_get_solve_info);
                               pbng_sweep rejects it.                              */
    double gamma;           /* Chebyshev relaxation (1.7)                          */
    double step;            /* scale of the Newton step of Eq. pbgn_dx (1.0)       */
    double skip_tol;        /* skip nodes with |r_i| <= skip_tol; 0 = never skip   */
    int32_t residual_every; /* pbng_solve: sweeps between residual checks (>= 1)   */
    int32_t resume;         /* 1: continue from the handle's iterate, its
                               acceleration history and sweep index; u_dev is
                               then output only.  0: start from u_dev.             */
    int32_t precision;      /* PBNG_PREC_*: FP32, COMPENSATED (the iterate is a
                               float32 pair, hi + lo; neighbour differences and
                               updates are formed in that pair; element
                               arithmetic float32), EXTENDED or AUTO (see the
                               enum)                                              */
    int32_t kernel_path;    /* 0: 1-ring layout kernels (TMA-staged records,
                               cp.async 1-ring gathers) for every colour whose
                               vertices have at most 32 incident tets and 32
                               1-ring vertices, CSR direct loads for the others;
                               1: CSR direct-load kernels everywhere.  Changing it
                               rebuilds the layout.                               */
    int32_t colour_order;   /* PBNG_ORDER_FORWARD: one sweep runs the colour
                               passes 0..C-1 (Section "Coloring and
                               Parallelism").  PBNG_ORDER_SYMMETRIC: 0..C-1 and
                               then C-2..0 (2C - 1 passes), the palindromic
                               order of symmetric Gauss-Seidel.  The paper does
                               not fix the order of the colour loop.  Linearised
                               at an equilibrium, the symmetric sweep is
                               self-adjoint in the Hessian's inner product, with
                               real eigenvalues in [0, 1) where the modified
                               nodal Hessian dominates the true diagonal block:
                               the spectrum the Chebyshev weights assume.  The
                               ascending order's eigenvalues are complex.  Also
                               the order of the adjoint's block Gauss-Seidel.   */
    int32_t reserved[2];
} pbng_params;

enum { PBNG_ORDER_FORWARD = 0, PBNG_ORDER_SYMMETRIC = 1 };

/* Fills p with the paper's defaults: corotated, no acceleration, omega 1.7,
 * rho 0.95, gamma 1.7, step 1, skip_tol 0, residual_every 10, resume 0,
 * compensated precision, kernel_path 0, forward colour order. */
void pbng_default_params(pbng_params* p);

/* Creates a mesh handle (Section "Discretization": P1 tetrahedra, per-tet
 * constant dN/dX and rest volume V^0; Eq. lame for (mu, lambda)).
 *   rest_xyz  host double [nv][3]  rest positions X
 *   tets      host int32  [ne][4]  vertex ids (either orientation)
 *   young     host double [ne]     Young's modulus E_e > 0
 *   poisson   host double [ne]     Poisson ratio, 0 <= nu < 0.5
 *   mesh_id   host int32  [nv] or NULL: component id of each vertex for
 *             batches of independent meshes (ids 0..ncomp-1); NULL = one mesh
 *   stream    cudaStream_t as void*, or NULL for the legacy default stream
 * The device is the one current at this call.  Fails with PBNG_EDEGENERATE if
 * a rest tet has |det Dm|/6 <= 1e-12 h^3 (h = its largest edge component),
 * PBNG_EINVAL on bad ids or sizes. */
pbng_status pbng_create_mesh(const double* rest_xyz, int32_t nv, const int32_t* tets, int32_t ne,
                             const double* young, const double* poisson, const int32_t* mesh_id,
                             void* stream, pbng_mesh** out);

/* Sets the boundary data (replaces earlier calls).  Eq. fem_d: clamped
 * vertices dir_idx[nd] are held at dir_xyz (host double [nd][3], absolute
 * positions).  Section "Weak Constraints": springs tie vertex spr_idx[s] to
 * spr_target[s] (host double [ns][3]) with energy spr_k[s]/2 |x - t|^2.
 * plane_nd (host double [4] = n, d, or NULL) adds contact energy
 * k_contact/2 (n.x - d)^2 for n.x < d (n is normalised by the library).
 * body_accel (host double [3] or NULL) with density (host double [ne], or
 * NULL = 1) gives f^ext_i = sum_e rho_e a V_e / 4.  Re-colours the free
 * vertices (Dirichlet vertices take no colour). */
pbng_status pbng_set_constraints(pbng_mesh* m, const int32_t* dir_idx, const double* dir_xyz,
                                 int32_t nd, const int32_t* spr_idx, const double* spr_target,
                                 const double* spr_k, int32_t ns, const double* plane_nd,
                                 double k_contact, const double* body_accel,
                                 const double* density);

/* Per-component body acceleration (for batches whose meshes carry different
 * loads): accel host double [ncomp][3], density host double [ne] or NULL
 * (= 1).  Replaces the body force of pbng_set_constraints; f^ext_i =
 * sum_e rho_e a_c V_e / 4 with c the component of tet e (Section
 * "Discretization").  Call after pbng_set_constraints. */
pbng_status pbng_set_body_accel(pbng_mesh* m, const double* accel, const double* density);

/* Replaces the per-tet material (host double [ne] each; Eq. lame for mu and
 * lambda).  The layout is rebuilt on the next call that needs it, and the
 * iterate history is dropped. */
pbng_status pbng_set_material(pbng_mesh* m, const double* young, const double* poisson);

/* Greedy node colouring of Section "Coloring and Parallelism": free vertices
 * in ascending id take the least colour not used by any vertex sharing a tet.
 * colour_out: host int32 [nv], -1 for clamped vertices.  ncolours: host. */
pbng_status pbng_get_colouring(pbng_mesh* m, int32_t* colour_out, int32_t* ncolours);

/* Runs nsweeps PBNG iterations on u_dev (device float [nv][3], in/out; the
 * entries of clamped vertices are overwritten with x_D - X).  If
 * rel_residual_out (host double[1] per component, or NULL) is given, the
 * FP64 relative residual |f + f^ext|_free / r_0 after the last sweep is
 * written, r_0 being the residual at the start (resume = 0) or the stored one.
 * Synchronises the stream before returning. */
pbng_status pbng_sweep(pbng_mesh* m, float* u_dev, int32_t nsweeps, const pbng_params* p,
                       double* rel_residual_out);

/* pbng_sweep from and to host memory, in one round trip: copies u_host
 * (host float [nv][3], in/out; pinned memory makes the copies asynchronous)
 * to a device buffer of the handle, loads it (p->resume is ignored: every
 * call starts a fresh acceleration history), runs nsweeps iterations as
 * pbng_sweep does, and copies the iterate back with the clamped entries set
 * to x_D - X.  If residual_out (host double [ncomp], or NULL) is given, the
 * FP64 absolute residual |f + f^ext|_free of each component after the last
 * sweep is written: the step's metric, which needs no residual at the
 * start.  Everything is enqueued on the handle's stream and the call
 * synchronises once, at the end. */
pbng_status pbng_sweep_host(pbng_mesh* m, float* u_host, int32_t nsweeps, const pbng_params* p,
                            double* residual_out);

/* Sweeps until every component's relative residual is <= rel_tol (checked
 * every p->residual_every sweeps) or max_sweeps is reached.  sweeps_out (host,
 * may be NULL) receives the sweeps done; rel_residual_out (host double
 * [ncomp], may be NULL) the final relative residuals.  Returns
 * PBNG_ENOTCONVERGED when max_sweeps ran out, PBNG_EDIVERGED when a check
 * finds a component's residual non-finite, above 1e3 r_0, or above r_0 and
 * 100 times the smallest residual of that component in this solve (sustained
 * growth).  On every exit, errors included, each component of a batch is
 * left active for later calls. */
pbng_status pbng_solve(pbng_mesh* m, float* u_dev, double rel_tol, int32_t max_sweeps,
                       const pbng_params* p, int32_t* sweeps_out, double* rel_residual_out);

/* Equilibrium adjoint (sensitivities of a loss L(u) of the equilibrium with
 * respect to per-tet log E and the clamped positions).  The paper states the
 * forward problem (Eq. fem_qs / Eq. fem_d) and the true nodal Hessian
 * (Eq. hess); the adjoint follows from differentiating fem_qs: with
 * H = -d(f + f^ext)/dx over free vertices at the equilibrium u_eq,
 *   H lambda = dL/du (free vertices),
 *   dL/dlog E_e = -sum_{i in e, free} lambda_i . V_e P(F_e) g_i,
 *   dL/dx_D = dL/du_D - H_DF lambda.
 * lambda is found with the same colour-by-colour block Gauss-Seidel as the
 * forward sweep (true Hessian applied matrix-free, 3x3 diagonal blocks
 * solved exactly), in p->colour_order, with p->accel acceleration
 * (Chebyshev with rho <= 0: the automatic rho of pbng_solve, measured on
 * this iteration), until |dL/du - H lambda| <= rel_tol |dL/du| or
 * max_sweeps.  With the symmetric order the iteration is symmetric block
 * Gauss-Seidel on H, whose spectrum is real in [0, 1) at a stable
 * equilibrium (H positive definite).
 * PBNG_ACCEL_CG (with PBNG_ORDER_SYMMETRIC only; EINVAL otherwise) uses the
 * same sweep as the preconditioner of conjugate gradients instead of as a
 * stationary iteration: each iteration runs one symmetric sweep from zero
 * on the current residual (z = M^{-1} r with M = (D + L) D^{-1} (D + L^T),
 * symmetric positive definite with H) and one matrix-free Hessian action,
 * and counts as one sweep in max_sweeps and sweeps_out; a direction of
 * non-positive curvature (H not positive definite) returns PBNG_EDIVERGED.
 * Its residual is the recursive one of the iteration, read back every 8
 * iterations (so a solve may run up to 7 iterations past its tolerance);
 * with float32 precision the true residual is evaluated at the end and
 * reported.
 * Precision: the sweeps are float32 (multipliers and the Hessian action);
 * their relative residual stalls near 1e-7 (L/h)^2 on a mesh of L/h
 * elements across (2e-3 at 48^3 with Chebyshev).  With p->precision
 * PBNG_PREC_EXTENDED or PBNG_PREC_AUTO the solve is refined instead: the
 * multipliers accumulate as float pairs, each correction solves
 * H d = dL/du - H lambda with the float32 sweeps (to 1e-2 of its right-hand
 * side, 1e-3 with PBNG_ACCEL_CG, or only to half of what is left to rel_tol
 * when that is less, or to their floor), and the residual is formed by
 * central differences
 * of the float-float force (PBNG_PREC_EXTENDED),
 * H lambda = -(F(u + eps lambda) - F(u - eps lambda)) / (2 eps), with
 * eps |lambda|_max = 1e-4 of the smallest element size; rel_tol then applies
 * to that residual.  max_sweeps counts the sweeps of all corrections.
 *   u_eq_dev      device float [nv][3]  equilibrium displacement (input)
 *   dLdu_dev      device float [nv][3]  dL/du (caller order; clamped rows are dL/dx_D)
 *   dL_dlogE_dev  device float [ne]     output, caller tet order
 *   dL_dxD_dev    device float [nd][3]  output, in the dir_idx order of
 *                                       pbng_set_constraints (may be NULL)
 * Requires every colour in the ring layout (vertices with at most 32
 * incident tets and 1-ring vertices) and kernel_path 0.  H must be positive
 * definite (a stable equilibrium); otherwise the iteration diverges
 * (PBNG_EDIVERGED) or a diagonal block is singular (PBNG_EDEGENERATE).
 * sweeps_out and rel_residual_out (host, may be NULL).  Synchronises. */
pbng_status pbng_adjoint(pbng_mesh* m, const float* u_eq_dev, const float* dLdu_dev, float* dL_dlogE_dev,
                         float* dL_dxD_dev, double rel_tol, int32_t max_sweeps, const pbng_params* p,
                         int32_t* sweeps_out, double* rel_residual_out);

/* General weak constraints (Section "Weak Constraints"): constraint c adds
 * (1/2) C_c^T K_c C_c to the energy, C_c(y) = sum_j w0_cj y_j - sum_j w1_cj y_j
 * joining two interpolated points (zero rest length), and
 * K_c = k_tau I + (k_n - k_tau) n n^T (n normalised here).
 *   idx     host int32 [nc][8]: side 0 in columns 0..3, side 1 in 4..7,
 *           -1 = unused (a vertex may appear on both sides)
 *   w       host double [nc][8]: weights >= 0, each side summing to one
 *   kn, kt  host double [nc] >= 0;  normal  host double [nc][3], nonzero
 * Each node update adds -beta K_c C_c to its force and beta^2 K_c to its
 * nodal Hessian (beta = w0 - w1 at the node; Eq. mod_hess).  The colouring
 * treats each constraint like an element (its free vertices get distinct
 * colours).  recolour = 0 colours the mesh again from scratch; 1 keeps the
 * current colours and revisits only the constraint vertices (Section
 * "Collision Coloring": a vertex keeps its colour unless a neighbour through
 * a tet or a constraint uses it, else takes the least unused colour), so
 * adding constraints to a coloured mesh recolours only their vertices.
 * The layout is rebuilt on the next call (pbng_get_profile reports the
 * colouring and layout times).  nc = 0 removes all constraints.  A
 * constraint may not join two batch components.  pbng_adjoint, pbng_force,
 * pbng_hessian_apply and pbng_newton_cg include the constraints (their true
 * Hessian blocks beta_i beta_j K_c; a constraint's clamped vertices enter
 * dL/dx_D). */
pbng_status pbng_set_weak_constraints(pbng_mesh* m, int32_t nc, const int32_t* idx, const double* w,
                                      const double* kn, const double* kt, const double* normal, int32_t recolour);

/* Backward Euler (Section "Position-Based Dynamics", Eq. fem_be): with
 * dt > 0 each free vertex gains the inertial term -m_ii (x_i - xhat_i) / dt^2
 * in its force and m_ii / dt^2 on the diagonal of its nodal Hessian, i.e. a
 * zero-rest-length spring of stiffness m_ii / dt^2 to the inertial target
 * xhat = 2 x^n - x^{n-1}; PBNG then minimises the incremental potential of one
 * time step.  The mass is lumped: m_ii = sum_e density_e V_e / 4 (the
 * integral of R^0 N_i for P1 tets).
 *   density  host double [ne], > 0 (required when dt > 0)
 * dt <= 0 returns the handle to quasistatics.  The layout is rebuilt on the
 * next call; until pbng_step sets it, xhat is the rest position. */
pbng_status pbng_set_inertia(pbng_mesh* m, double dt, const double* density);

/* One backward-Euler time step (needs pbng_set_inertia with dt > 0).
 *   u_dev       device float [nv][3]: u^n on entry, u^{n+1} on return
 *   u_prev_dev  device float [nv][3]: u^{n-1} on entry, u^n on return
 * A kernel sets xhat = 2 u^n - u^{n-1} and the initial guess
 * xhat + dt^2 f^ext_i / m_ii (the predictor the paper describes for PBD;
 * the initial guess only changes the first iterates), then the step runs
 * as pbng_solve(rel_tol, max_sweeps = nsweeps) when rel_tol > 0, else as
 * nsweeps sweeps of pbng_sweep; resume is ignored (every step starts a
 * fresh acceleration history).  Clamped vertices take their current targets
 * (pbng_set_dirichlet_targets).  sweeps_out and rel_residual_out (host, per
 * component) may be NULL. */
pbng_status pbng_step(pbng_mesh* m, float* u_dev, float* u_prev_dev, int32_t nsweeps, double rel_tol,
                      const pbng_params* p, int32_t* sweeps_out, double* rel_residual_out);

/* New targets for the clamped vertices of the last pbng_set_constraints
 * (host double [nd][3], in its dir_idx order) without rebuilding the layout:
 * for animated boundaries.  They apply when the iterate is next loaded (a
 * call with resume = 0, or pbng_step).  Synchronises. */
pbng_status pbng_set_dirichlet_targets(pbng_mesh* m, const double* dir_xyz);

/* Force and Hessian of the discrete energy (model p->model, kernel_path 0; p may
 * be NULL for the defaults), for Krylov or optimisation methods around PBNG.
 * pbng_force: f_out_dev (device float [nv][3]) = f(u) + f^ext on free
 *   vertices (the force of Eq. fem_qs with the weak terms; zero rows at
 *   clamped vertices).
 * pbng_hessian_apply: hp_out_dev = H p on free vertices, H = -d(f + f^ext)/du
 *   the true Hessian (Eq. hess, with dR of the polar factor) at u, p_dev a
 *   direction (rows of clamped vertices ignored; zero rows on output).
 * All arrays device float [nv][3] in caller order.  Synchronise. */
pbng_status pbng_force(pbng_mesh* m, const float* u_dev, const pbng_params* p, float* f_out_dev);
pbng_status pbng_hessian_apply(pbng_mesh* m, const float* u_dev, const float* p_dev, const pbng_params* p,
                               float* hp_out_dev);

/* Newton-CG reference solver on the same GPU (the paper compares PBNG with
 * Newton's method; Section "PBNG vs. PBD and Limited Newton"): each Newton
 * iteration solves H dx = f + f^ext with block-Jacobi preconditioned CG on the
 * true Hessian (pbng_hessian_apply), stopping at |r_cg| <= cg_tol |f + f^ext|,
 * after max_cg iterations or at the first direction of non-positive
 * curvature; a backtracking line search halves the step until the residual
 * norm decreases; if none is accepted, the preconditioned residual is tried
 * once.  Stops at |f + f^ext| <= rel_tol r_0 (global 2-norm over all
 * components, r_0 at u_dev) or max_newton iterations (PBNG_ENOTCONVERGED).
 * Any model (p->model); kernel_path 0 only.  u_dev in / out.  info may be NULL.
 * The acceleration history of the handle is reset.  Synchronises. */
typedef struct {
    int32_t newton_iterations;
    int32_t cg_iterations;          /* summed over Newton iterations            */
    int32_t line_search_halvings;
    int32_t fallbacks;              /* steps along the preconditioned residual  */
    double rel_residual;            /* |f + f^ext| / r_0 at the end              */
} pbng_newton_info;
pbng_status pbng_newton_cg(pbng_mesh* m, float* u_dev, double rel_tol, int32_t max_newton, int32_t max_cg,
                           double cg_tol, const pbng_params* p, pbng_newton_info* info);

/* Checkpoint of the iteration: the iterate (float32 pairs), the two previous
 * iterates used by the acceleration, the sweep index, omega_l and r_0.
 * pbng_get_state with buf == NULL writes the size needed to *bytes;
 * otherwise it copies the state into buf (host, *bytes large enough) and
 * sets *bytes.  pbng_set_state restores it into a handle built from the same
 * mesh and constraints (same layout; PBNG_EINVAL otherwise); the next
 * pbng_sweep / pbng_solve with resume = 1 then continues bit for bit as if
 * the iteration had never stopped.  Both synchronise. */
pbng_status pbng_get_state(pbng_mesh* m, void* buf, size_t* bytes);
pbng_status pbng_set_state(pbng_mesh* m, const void* buf, size_t bytes);

/* FP64 2-norm of (f + f^ext) over free vertices at u_dev (Section "PBNG vs.
 * PBD and Limited Newton": the 2-norm of the Newton residual), per component
 * (host double [ncomp]).  The element forces are evaluated in float-float
 * arithmetic (as PBNG_PREC_EXTENDED) when every colour is in the ring layout,
 * else in float32; each vertex's sum in FP64.  Does not modify u_dev. */
pbng_status pbng_residual(pbng_mesh* m, const float* u_dev, double* residual_out);

/* pbng_residual without any allocation.  The paper has no counterpart: this
 * is a service of the library for callers that must not allocate memory once
 * their solve loop is running — for example an application whose GPU memory
 * is entirely handed to its own pool allocator, or a real-time loop in which a
 * cudaMalloc or cudaFree (either can synchronise the whole device) is not
 * allowed.  It computes the same per-component FP64 residual norms as
 * pbng_residual with the same kernels, but calls no cudaMalloc, cudaFree or
 * other allocating routine, on the device or the host (its error texts go
 * into a buffer the handle reserves when it is created; only the text of a
 * PBNG_ECUDA failure, after which the handle is unusable, may take host
 * memory).
 *   - Its FP64 partial sums live in one fixed array of 65,536 doubles
 *     (512 KiB) that the library reserves on every GPU that loads it, until
 *     the process exits.  A mesh whose residual launch needs more partial
 *     sums (one per 256-thread block; beyond roughly 20 million incidences)
 *     or has more than 65,536 components is rejected with PBNG_EINVAL.
 *   - The handle's layout must exist already: make any pbng_get_colouring,
 *     pbng_sweep, pbng_solve or pbng_residual call after the last
 *     pbng_set_constraints first (layout building allocates); otherwise
 *     PBNG_EINVAL.
 *   - The first call on a device looks the array's device address up once
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Every call, from any handle or thread, uses the same array and leaves
 *     its last contents there; calls whose GPU work overlaps (different
 *     streams or threads at the same time) race and return wrong sums.
 *   - Synchronises the handle's stream; writes residual_out (host double
 *     [ncomp]).  u_dev as for pbng_residual. */
pbng_status pbng_residual_noalloc(pbng_mesh* m, const float* u_dev, double* residual_out);

/* Per-kernel timing on the handle's stream (tracing; Section "Coloring and
 * Parallelism" reports per-iteration runtimes).  While enabled, each colour
 * pass, acceleration and residual launch is bracketed by CUDA events.
 * Counters accumulate from the pbng_set_profiling(m, 1) call. */
typedef struct {
    int64_t colour_pass_launches;
    double colour_pass_ms;        /* summed event time of all colour passes   */
    int64_t accel_launches;
    double accel_ms;
    int64_t residual_launches;    /* residual evaluations (all colours + sum) */
    double residual_ms;
    int64_t kernel_launches;      /* every kernel this handle launched        */
    int64_t free_vertices;        /* of the current layout                    */
    int64_t incidences;           /* (free vertex, incident tet) pairs        */
    int32_t ncolours;
    int32_t reserved;
    double colour_ms;             /* host time of the last colouring (or recolouring) */
    double layout_ms;             /* host time of the last layout build, colouring included */
} pbng_profile;

/* enable = 1 starts (and zeroes) the counters, 0 stops timing. */
pbng_status pbng_set_profiling(pbng_mesh* m, int32_t enable);

/* Test hook for the device-side timeouts.  Every wait of the ring passes on
 * an asynchronous copy gives up after about two seconds of SM clock, records
 * kErrTimeout and lets the warp's other copies land before it returns; the
 * call then fails with PBNG_ETIMEOUT.  With bytes > 0 (a multiple of 16, at
 * most 1024) each warp's first bulk copy of every later ring pass (an
 * item's records; in the float32 passes, its 1-ring ids) is expected to
 * carry that many bytes more than it does, so that wait runs out
 * while every copy still completes.  0 restores normal operation.  Drops the
 * captured sweep graphs; EINVAL on a bad value. */
pbng_status pbng_test_set_copy_shortfall(pbng_mesh* m, int32_t bytes);
/* Synchronises the stream and returns the counters. */
pbng_status pbng_get_profile(pbng_mesh* m, pbng_profile* out);

/* Launch schedules of the 1-ring colour passes (kernel_path 0).  The paper
 * runs each colour as one parallel loop (Section "Coloring and
 * Parallelism"); here each colour is one launch of a persistent grid whose
 * warps stream 32-lane work items, and three knobs decide how:
 *   ctas_per_sm  1..PBNG_MAX_CTAS_PER_SM CTAs (8 warps each) per SM
 *   blocked      0: warp w takes items w, w + nwarps, ... (strided);
 *                1: warp w takes one contiguous run of items (blocked)
 *   balanced     1: the grid is trimmed to the fewest CTAs whose warps still
 *                finish in the same number of item rounds (no warp idles
 *                through the last round); 0: the full grid
 * The vertex updates of one colour are independent, so every schedule gives
 * a bit-identical iterate; only the time differs.  Colours laid out for
 * direct loads (vertices with more than 32 incident tets or 1-ring vertices,
 * or kernel_path 1) have no schedule and report ctas_per_sm = 0. */
#define PBNG_MAX_COLOURS 64
#define PBNG_MAX_CTAS_PER_SM 2
typedef struct {
    int32_t ncolours;                          /* of the current layout       */
    int32_t ctas_per_sm[PBNG_MAX_COLOURS];     /* per colour; 0 = not a ring colour */
    int32_t blocked[PBNG_MAX_COLOURS];
    int32_t balanced[PBNG_MAX_COLOURS];        /* 1: grid trimmed to the fewest
                                                  warps taking the same number
                                                  of item rounds            */
    double default_ms_per_sweep;   /* pbng_autotune: colour passes of one sweep
                                      with the default schedule (3, strided)   */
    double tuned_ms_per_sweep;     /* ... with the schedule it chose           */
    int32_t candidates;            /* schedules timed per colour               */
    int32_t reserved;
} pbng_schedule;

/* Sets the schedule of every ring colour from s->ctas_per_sm[c] (clamped to
 * 1..PBNG_MAX_CTAS_PER_SM), s->blocked[c] and s->balanced[c] for
 * c < min(s->ncolours, ncolours of the layout).  Builds the layout if needed (p selects
 * kernel_path; NULL = defaults).  Captured sweep graphs are dropped and
 * re-captured on next use.  The schedule survives layout rebuilds that keep
 * the colour count. */
pbng_status pbng_set_schedule(pbng_mesh* m, const pbng_params* p, const pbng_schedule* s);
/* Current schedule (ms fields = 0 unless set by pbng_autotune). */
pbng_status pbng_get_schedule(pbng_mesh* m, pbng_schedule* out);

/* Autotuner: times every schedule (ctas_per_sm x {strided, blocked} x
 * {full, balanced grid}) of every
 * ring colour over `reps` sweeps each, on a scratch copy of u_dev (the
 * caller's u_dev, the handle's iterate and its acceleration history are not
 * touched) and keeps the fastest per colour (the default unless another is
 * at least 2 % faster).  The candidates alternate: each of the `reps` rounds
 * runs every candidate once over all colours, each colour pass bracketed by
 * CUDA events on the handle's stream.  out (may be NULL) receives the chosen
 * schedule and the summed colour-pass time per sweep of the default and of
 * the chosen schedules from the same rounds.  Synchronises; reps in 1..1000. */
pbng_status pbng_autotune(pbng_mesh* m, const float* u_dev, const pbng_params* p, int32_t reps,
                          pbng_schedule* out);

/* What the last pbng_solve ran with.  With automatic rho (Chebyshev,
 * rho <= 0) pbng_solve first runs max(30, 3 residual_every) plain sweeps,
 * takes the per-sweep contraction q = (r_b / r_a)^(1 / (b - a)) of the
 * slowest active component between the residual check a at or after a third
 * of them and the last one b, and restarts the Chebyshev schedule
 * (omega_1 = omega_2 = 1, x^{-1} = x^0) at the current iterate with
 *   forward order:   rho = clamp(1 - 2 (1 - q), 0.5, 0.98).  The Chebyshev
 *                    weights assume error modes that decay with real factors
 *                    up to rho; colour-ordered Gauss-Seidel on more than two
 *                    colours does not guarantee that, and a rho at the
 *                    measured rate itself can diverge, hence the factor 2 and
 *                    the cap;
 *   symmetric order: rho = clamp(1 - gamma (1 - q), 0.5, 1 - 1e-6), the
 *                    spectral radius of gamma B + (1 - gamma) I for a real
 *                    spectrum of B in [0, q].  A few plain sweeps underrate
 *                    the slowest mode, so once a window of
 *                    max(4 residual_every, 3 / sqrt(2 (1 - rho))) sweeps has
 *                    passed since the last (re)start, an observed per-sweep
 *                    factor f (over its second half) that lowered the
 *                    residual below 0.8 of its value (after a first half
 *                    that lowered it below 0.9) but at under 70 % of the
 *                    log-rate of k = rho / (1 + sqrt(1 - rho^2)) raises rho
 *                    to rho (z + 1/z) / 2, z = f / k (where a mode above
 *                    rho sits), and restarts (at most 12 raises).
 * A residual check whose worst component exceeds 4x the best seen since the
 * last (re)start doubles 1 - rho and restarts the schedule; after 4 such
 * back-offs the remaining sweeps are plain.  The estimate is not kept across
 * calls. */
#define PBNG_MAX_SOLVE_EVENTS 16
typedef struct {
    double rho;              /* Chebyshev rho in use at the end (0: none)     */
    double plain_rate;       /* automatic rho: measured q; else 0              */
    int32_t estimate_sweeps; /* automatic rho: plain sweeps before Chebyshev   */
    int32_t restarts;        /* automatic rho: divergence back-offs            */
    int32_t raises;          /* automatic rho, symmetric order: rho raises     */
    int32_t extended_from;   /* sweeps done before the colour passes ran in
                                PBNG_PREC_EXTENDED (0 for EXTENDED, the stall
                                point for AUTO); -1: never                    */
    int32_t nevents;         /* automatic rho: schedule (re)starts recorded    */
    int32_t event_sweep[PBNG_MAX_SOLVE_EVENTS];  /* sweeps done at each (re)start */
    double event_rho[PBNG_MAX_SOLVE_EVENTS];     /* its rho (0: plain from there) */
} pbng_solve_info;
pbng_status pbng_get_solve_info(const pbng_mesh* m, pbng_solve_info* out);

/* Measurement aid (no counterpart in the paper): the FP32 FMA throughput of
 * the current device in TFLOP/s (one FMA = 2 flops), the denominator of the
 * float32 element arithmetic's roofline.  Runs 6 launches of 8 CTAs of 256
 * threads per SM, each thread carrying 8 independent FMA chains for 32,768
 * rounds, timed with CUDA events on `stream` (cudaStream_t as void*, NULL =
 * legacy default stream); reports the best of the last 5.  Allocates and
 * frees a small output buffer; changes no device setting.  Synchronises. */
pbng_status pbng_measure_fp32_peak(void* stream, double* tflops_out);

/* Number of independent components (1 unless mesh_id was given). */
int32_t pbng_num_components(const pbng_mesh* m);

const char* pbng_status_string(pbng_status s);
/* Text of the last failure on this handle ("" if none); valid until the next call. */
const char* pbng_last_error(const pbng_mesh* m);
void pbng_destroy(pbng_mesh* m);

#ifdef __cplusplus
}
#endif
#endif /* PBNG_H */
