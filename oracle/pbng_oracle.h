/*
 * PBNG FP64 oracle — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, serial (optionally OpenMP over the vertices of one colour, which
 * gives bit-identical results), obviously-correct double-precision restatement
 * of Position-Based Nonlinear Gauss-Seidel (Chen, Han, Chen, Teran,
 * arXiv 2306.09021).  Only tests/, the smoke check and the benchmark's CPU
 * baseline leg call it.  It shares no code with the CUDA library.
 *
 * Conventions: 3x3 matrices are row-major double[9]; positions are absolute
 * (x, not displacement), double[3*nv]; gradients g_j = dN_j/dX are the rows of
 * B = Dm^{-1} for j = 1..3 and g_0 = -(g_1+g_2+g_3).
 */
#ifndef PBNG_ORACLE_H
#define PBNG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Eq. (lame): mu = E/(2(1+nu)), lambda = E nu / ((1+nu)(1-2nu)). */
void ora_lame(double E, double nu, double* mu, double* lam);

/* One-sided Jacobi SVD F = U diag(s) V^T, s descending, U, V orthogonal.
 * Returns the number of Jacobi sweeps used. */
int ora_svd3(const double* F, double* U, double* s, double* V);

/* Rotation R in SO(3) of the polar decomposition used by the corotated model
 * (Eq. cor): R = U diag(1,1,det(U V^T)) V^T, i.e. the smallest singular value
 * takes the sign of det F.  shat (may be NULL) receives the signed values. */
void ora_polar(const double* F, double* R, double* shat);

/* Energy density of model 0 fixed corotated (Eq. cor), 1 Neo-Hookean
 * (Eq. nh, lambda_hat = mu + lambda) or 2 stable Neo-Hookean (Eq. snh, with
 * lambda on its volume term and Smith et al.'s mu' = 4mu/3,
 * lambda' = lambda + 5mu/6, alpha = 1 + 3mu'/(4lambda')); mu, lambda are the
 * Lame parameters of Eq. lame. */
double ora_psi(const double* F, double mu, double lam, int model);
/* First Piola-Kirchhoff stress P = dPsi/dF of the model. */
void ora_pk1(const double* F, double mu, double lam, int model, double* P);
/* True energy-density Hessian of the model applied to dF (Newton, adjoint). */
void ora_dpk1(const double* F, const double* dF, double mu, double lam, int model, double* dP);
/* Modified density Hessian, Eq. (mod_hess_dens):
 * C[(a*3+g)*9 + (b*3+d)] = 2mu d_ab d_gd + lam cof(F)_ag cof(F)_bd. */
void ora_modified_density_hessian(const double* F, double mu, double lam, double* C81);
/* Cofactor matrix det(F) F^{-T}, defined for every F. */
void ora_cofactor(const double* F, double* C);

/* Mesh + boundary data.  Copies every input.  status: 0 ok, 1 invalid input,
 * 4 degenerate rest tetrahedron.  is_dir[nv] marks clamped vertices, whose
 * positions are whatever the caller puts in x.  body_accel[3] and density[ne]
 * may be NULL.  Springs tie vertex spr_idx[s] to spr_t[3s..] with stiffness
 * spr_k[s] (energy k/2 |x-t|^2).  plane[4] = (n, d) or NULL: a vertex with
 * n.x < d gets energy k_contact/2 (n.x-d)^2. */
void* ora_create(int nv, const double* X, int ne, const int* tets,
                 const double* young, const double* poisson,
                 const unsigned char* is_dir,
                 const double* body_accel, const double* density,
                 int ns, const int* spr_idx, const double* spr_t, const double* spr_k,
                 const double* plane, double k_contact, int* status);
void ora_destroy(void* h);
/* Constitutive model of the mesh (0, 1, 2 as for ora_psi; default 0).  The
 * modified Hessian of Eq. mod_hess_dens is the same for every model.
 * Returns nonzero for an unknown model. */
int ora_set_model(void* h, int model);
/* Order of the colour passes inside one sweep (ora_sweeps).  0: ascending,
 * colours 0..C-1 (Section "Coloring and Parallelism"; the default).
 * 1: symmetric, colours 0..C-1 and then C-2..0 (2C - 1 passes), the
 * palindromic order of symmetric Gauss-Seidel; the paper does not fix the
 * order of the colour loop.  Returns nonzero for another value. */
int ora_set_colour_order(void* h, int order);
/* Backward Euler (Eq. fem_be): with dt > 0 every free vertex gets the
 * inertial term -m_ii (x_i - xhat_i) / dt^2 in its force, m_ii / dt^2 on the
 * diagonal of its Hessian and (m_ii / 2 dt^2)|x_i - xhat_i|^2 in the energy,
 * with the lumped mass m_ii = sum_e density_e V_e / 4.  xhat (absolute
 * [nv][3]) is the inertial target 2 x^n - x^{n-1}.  dt <= 0 turns it off.
 * Returns nonzero on a NULL array. */
int ora_set_inertia(void* h, double dt, const double* density, const double* xhat);
/* General weak constraints (Section "Weak Constraints"):
 * C_c(y) = sum_j w0_cj y_j - sum_j w1_cj y_j, energy (1/2) C_c^T K_c C_c with
 * K_c = kt_c I + (kn_c - kt_c) n_c n_c^T.  Constraint c lists up to four
 * nodes per side in idx[8c .. 8c+3] (side 0) and idx[8c+4 .. 8c+7] (side 1),
 * -1 = unused, with non-negative weights w summing to one per side.  The
 * colouring treats each constraint like an element; recolour = 1 keeps the
 * current colours and revisits only the constraint nodes (Section
 * "Collision Coloring"), 0 colours every node again.  Nonzero on bad input. */
int ora_set_weak_constraints(void* h, int nc, const int* idx, const double* w, const double* kn, const double* kt,
                             const double* nrm, int recolour);
/* The lumped masses of the last ora_set_inertia (0 before). */
void ora_lumped_mass(const void* h, double* out);

/* Greedy node colouring of Section "Coloring and Parallelism". */
int ora_num_colours(const void* h);
void ora_get_colours(const void* h, int* colour /* [nv], -1 = clamped */);
void ora_get_tet_constants(const void* h, double* B9, double* V, double* mu, double* lam);
void ora_get_fext(const void* h, double* fext3);

/* Local right-hand side r = f_i + f^ext_i and modified Hessian A_i (Eq.
 * pbgn_dx, Eq. mod_hess) of vertex i at positions x. */
void ora_local_system(const void* h, const double* x, int i, double* r3, double* A9);

/* Residual vector (f + f^ext) over free vertices (zero at clamped ones) and
 * its 2-norm.  r_out may be NULL. */
double ora_residual(const void* h, const double* x, double* r_out);
/* Total potential sum V Psi + weak/contact energy - sum f^ext . x. */
double ora_energy(const void* h, const double* x);

/* nsweeps PBNG sweeps in place on x, colours in the order of
 * ora_set_colour_order.  accel: 0 plain, 1 Chebyshev (rho,
 * gamma), 2 SOR (omega), both applied after each whole sweep with
 * x^{-1} = x^0.  skip_tol > 0 skips vertices with |r| <= skip_tol.
 * res_hist (NULL or nsweeps+1 doubles) receives |r| before and after every
 * sweep.  Returns 0, or 5 when a non-finite value appeared. */
int ora_sweeps(const void* h, double* x, int nsweeps, int accel, double omega,
               double rho, double gamma, double skip_tol, int nthreads, double* res_hist);

/* Newton's method with the true Hessian, dense LU and a backtracking line
 * search on the energy (tiny meshes only).  Returns iterations used, or -1
 * when the tolerance was not met. */
int ora_newton(const void* h, double* x, double rel_tol, int maxit, double* res_out);

/* Dense true Hessian -d(f + f^ext)/dx over all 3nv DOFs (row-major). */
void ora_hessian_dense(const void* h, const double* x, double* H);

/* Dense adjoint at an equilibrium x: solve H_FF lam = dL/dx_F, then
 * dL/dlogE_e = -sum_{i in e, free} lam_i . V_e P_e g_i and
 * dL/dx_D = dL/dx_D - H_DF lam (nd = number of clamped vertices, ascending id).
 * Returns 0 or 1 when H_FF is singular. */
int ora_adjoint_dense(const void* h, const double* x, const double* dLdx,
                      double* dLdlogE, double* dLdxD);

/* Threads ora_sweeps can use for nthreads requested (1 without OpenMP). */
int ora_threads_available(int nthreads);

#ifdef __cplusplus
}
#endif
#endif
