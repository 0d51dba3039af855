/*
 * Plain FP64 CPU oracle for the two-stage poromechanics preconditioner of
 * White, Castelletto, Klevtsov, Bui, Osei-Kuffuor, Tchelepi (arXiv 1812.05540).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may include, link or call this code.  Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline / reference legs use it.
 *
 * It restates, step by step and without blocking or fusion, what the paper
 * computes:
 *   - the Jacobian of the Q1-P0-P0 FE/FV discretisation (App. B) on a Cartesian
 *     box, with the residual of the weak form (§3, App. B) for finite-difference
 *     checks and the Terzaghi column;
 *   - the fixed-stress Schur approximation (§5.1), quasi-IMPES reduction (§5.3),
 *     smoothed-aggregation AMG for the SDC mechanics block (§5.2) and the
 *     pressure block (§5.3), block ILU(0) (§5.3, option 2), Algorithm 1;
 *   - flexible GMRES (right preconditioning, §4) with modified Gram-Schmidt;
 *   - dense LU with partial pivoting for brute-force checks.
 *
 * Memory returned by or_* functions is owned by the oracle and released with
 * the matching *_free call.  All indices are 0-based.
 */
#ifndef POROORACLE_H
#define POROORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* generator flags */
enum {
  OR_GRAVITY = 1 << 0,    /* body force and gravity in the flux potential */
  OR_DIRICHLET = 1 << 1,  /* base nodes fixed in all three components */
  OR_SCALE = 1 << 2,      /* block-row / pressure-column scaling (§4 remark) */
  OR_ACCUM = 1 << 3,      /* accumulation terms of the mass balances */
  OR_FLUX = 1 << 4,       /* TPFA face terms */
  OR_FLUX_SAT = 1 << 5,   /* saturation derivatives of the face fluxes */
  OR_COUPLING = 1 << 6,   /* A_uf and A_fu blocks */
  OR_ALL = 0x7f,          /* everything above; the wells below are an option */
  OR_WELLS = 1 << 7       /* Peaceman wells under bottom-hole pressure control (water injector, producer) */
};

/* field statistics */
enum { OR_FIELDS_LOGNORMAL = 0, OR_FIELDS_LAYERED = 1, OR_FIELDS_CHANNELS = 2,
       OR_FIELDS_HOMOGENEOUS = 3 };

typedef struct {
  int32_t nx, ny, nz;
  double h;              /* cubic cell edge [m] */
  uint64_t seed;
  int32_t field_kind;
  uint32_t flags;
  double dt;             /* [s] */
  double biot;
  double c_w, c_nw, c_r; /* compressibilities [1/Pa] */
  double mu_w, mu_nw;    /* [Pa s] */
  double rho_w0, rho_nw0, rho_s0;
  double s_wr, s_nwr;
  double grav;           /* [m/s^2] */
  double p_ref;          /* reference (initial formation) pressure [Pa] */
  double dp_amp;         /* amplitude of the smooth pressure perturbation [Pa] */
  double corey;          /* relative-permeability exponent (2 in §6) */
  /* homogeneous fields (field_kind == OR_FIELDS_HOMOGENEOUS) */
  double E0, nu0, kappa0, phi0, sw0;
  /* modulus of the fixed-stress diagonal (§5.1): 0 = drained bulk modulus K_dr (default), 1 = uniaxial
     (constrained) modulus K_dr + 4G/3 of the remark on one-dimensional loading */
  int32_t fs_modulus;
} or_gen_params;

typedef struct {
  int32_t nx, ny, nz;
  double h;
  int64_t n_nodes, n_cells, n_u, n_f, n;
  /* BSR, row-major blocks, sorted column indices */
  int64_t nnzb_uu, nnzb_uf, nnzb_fu, nnzb_ff;
  int64_t *uu_rp; int32_t *uu_ci; double *uu_v; /* 3x3, node x node */
  int64_t *uf_rp; int32_t *uf_ci; double *uf_v; /* 3x2, node x cell, cols (s,p) */
  int64_t *fu_rp; int32_t *fu_ci; double *fu_v; /* 2x3, cell x node, rows (s,p) */
  int64_t *ff_rp; int32_t *ff_ci; double *ff_v; /* 2x2, cell x cell */
  double *d_fs;        /* 2 per cell: (D_sp, D_pp), §5.1 */
  uint8_t *dirichlet;  /* per displacement dof */
  double *rhs;         /* n */
  double alpha_u, alpha_f;
  /* cell fields at the linearisation state */
  double *E, *nu, *kh, *kv, *phi0, *sw, *p;
} or_system;

/* host threads the row loops of this build use (1 unless built with -fopenmp) */
int or_num_threads(void);

/* splitmix64 output for the given state (Vigna's published generator) */
uint64_t or_splitmix64(uint64_t state);

/* unit-variance Gaussian random field (white noise convolved with exp(-(d/L)^2/2)) */
void or_correlated_field(uint64_t seed, int field, int nx, int ny, int nz, int Lx, int Ly, int Lz, double* out);

int or_generate(const or_gen_params* gp, or_system** out);
void or_system_free(or_system* s);
void or_default_params(or_gen_params* gp, int config);

/* y = A x over the full coupled Jacobian, x = [u (node-major xyz); (s,p) per cell] */
void or_spmv(const or_system* s, const double* x, double* y);

/* reference Q1 integrals on the cube of edge h (2x2x2 Gauss):
   G[8][8][3][3] = int dN_a/dx_d dN_b/dx_e, IN[8] = int N_a,
   IdN[8][3] = int dN_a/dx_d, INdN[8][8][3] = int N_a dN_b/dx_e */
void or_ref_integrals(double h, double* G, double* IN, double* IdN, double* INdN);

/* the system at the state base + dx (dx: n values ordered as x), the base state (u = 0, s = S_w, p of the
   fields) taken as the previous time level: the Jacobian there, Dirichlet elimination and scaling as in
   or_generate (alpha_u, alpha_f are that Jacobian's), rhs as in or_generate */
int or_generate_at(const or_gen_params* gp, const double* dx, or_system** out);

/* residual of the discrete weak form (§3, App. B) at x = state + dx, with the
   previous time level equal to the linearisation state (unscaled, no Dirichlet
   elimination).  Used for finite-difference checks of the Jacobian. */
int or_residual(const or_gen_params* gp, const double* dx, double* r);

/* preconditioner */
enum { OR_MECH_AMG = 0, OR_MECH_EXACT = 1, OR_MECH_AMG_RBM = 2 };  /* M_uu: SDC AMG, exact, rigid-body-mode SA */
enum { OR_FLOW_CPR = 0, OR_FLOW_EXACT_FS = 1, OR_FLOW_EXACT_SCHUR = 2 }; /* M_ff */
enum { OR_LOCAL_ILU0 = 0, OR_LOCAL_EXACT = 1, OR_LOCAL_GS = 2 }; /* M_L: ILU(0), exact, block Gauss-Seidel */
enum { OR_PRESS_AMG = 0, OR_PRESS_EXACT = 1 };                /* M_pp */
enum { OR_CPR_QUASI_IMPES = 0, OR_CPR_TRUE_IMPES = 1 };        /* D_ss, D_ps of the CPR reduction */
enum { OR_FS_GIVEN = 0, OR_FS_RSL = 1, OR_FS_RSL_EXACT = 2 };  /* D_sp, D_pp of S_ff^(FS) */

typedef struct {
  double theta_u, theta_p;
  int32_t coarse_max_u, coarse_max_p;
  int32_t max_levels;
  int32_t pre, post;
  int32_t smoother;     /* 0 = l1-Jacobi, 1 = Chebyshev on D^{-1}A */
  int32_t cheb_degree;
  double cheb_ratio;    /* Chebyshev interval [lambda_hat/ratio, lambda_hat] */
  int32_t mech_mode, flow_mode, local_mode, press_mode;
  int32_t full_exact; /* M^{-1} = A^{-1} (dense, tiny systems only) */
  int32_t local_sweeps; /* OR_LOCAL_GS: block Gauss-Seidel sweeps (3 in §6.1) */
  int32_t cpr_reduction; /* OR_CPR_QUASI_IMPES (diagonal entries) or OR_CPR_TRUE_IMPES (column sums), §5.3 */
  int32_t fs_mode;       /* fixed-stress diagonal of S_ff: OR_FS_GIVEN (the system's d_fs), OR_FS_RSL (row-sum
                            lumping of the §5.1 remark with one application of M_uu^{-1}), OR_FS_RSL_EXACT
                            (the same with A_uu^{-1} by dense LU; tiny systems) */
  int32_t ilu_tile_y, ilu_tile_z; /* OR_LOCAL_ILU0 scope: 0, 0 = global ILU(0); ty, tz > 0 = processor-local
                                     ILU(0) (§6: each process factors its own rows), the subdomains being the
                                     cell columns of ty x tz cells in (y, z) spanning x, i.e. the ILU(0) of
                                     S_ff with the blocks coupling different subdomains removed
                                     (default 16 x 8) */
} or_prec_params;

typedef struct or_prec or_prec;

void or_default_prec_params(or_prec_params* pp);
int or_prec_setup(const or_system* s, const or_prec_params* pp, or_prec** out);
/* the same with the mechanics AMG M_uu built from mech's A_uu (same grid): the flow-setup reuse of §5.4,
   where M_uu is built once and kept while the Jacobian changes from one Newton step to the next */
int or_prec_setup_reuse(const or_system* s, const or_system* mech, const or_prec_params* pp, or_prec** out);
void or_prec_free(or_prec* p);
void or_prec_apply(or_prec* p, const double* v, double* z);

/* hierarchy inspection: which = 0 mechanics, 1 pressure */
int or_amg_nlevels(const or_prec* p, int which);
int64_t or_amg_level_n(const or_prec* p, int which, int level);
int64_t or_amg_level_nnz(const or_prec* p, int which, int level);
/* copy out a level operator: rp[n+1], ci[nnz], v[ncomp*nnz] (component-major per entry) */
int or_amg_level_matrix(const or_prec* p, int which, int level, int64_t* rp, int32_t* ci, double* v);
/* aggregate of each row of level `level` (-1 = excluded); returns number of aggregates */
int64_t or_amg_aggregates(const or_prec* p, int which, int level, int32_t* agg);
/* 1 for the distance-2 MIS roots of level `level` */
int64_t or_amg_roots(const or_prec* p, int which, int level, uint8_t* root);
/* aggregation (strength graph, distance-2 MIS under the priority key of `level`, phase 1, phase 2) of a
   caller-given CSR operator with nc values per entry and sorted columns; agg[n] (-1 = not aggregated),
   root[n]; returns the number of aggregates */
int64_t or_aggregate(int64_t n, int nc, const int64_t* rp, const int32_t* ci, const double* v, double theta,
                     int level, int32_t* agg, uint8_t* root);
int64_t or_amg_p_nnz(const or_prec* p, int which, int level);
/* rigid-body-mode smoothed aggregation (OR_MECH_AMG_RBM) on the full A_uu: levels, and per level
   shape = {block rows n, block size b (3 finest, 6 below), block nnz, aggregates, P block nnz, coarsest},
   the b x b BSR operator, the aggregates agg[n], the near-nullspace B[n b][6], the tentative prolongator
   Pt[n b][6], the Gershgorin bound, and P as a b x 6 BSR; one V-cycle at the finest level */
int or_rbm_nlevels(const or_prec* p);
int or_rbm_level_shape(const or_prec* p, int level, int64_t* shape);
int or_rbm_level_matrix(const or_prec* p, int level, int64_t* rp, int32_t* ci, double* v);
int or_rbm_level_data(const or_prec* p, int level, int32_t* agg, double* B, double* Pt, double* lam);
int or_rbm_prolongator(const or_prec* p, int level, int64_t* rp, int32_t* ci, double* v);
int or_rbm_vcycle(const or_prec* p, const double* b, double* x);
/* the six rigid-body modes at the grid's nodes, node-major rows (x, y, z) of 6 */
void or_rigid_body_modes(int nx, int ny, int nz, double* B);
int or_amg_prolongator(const or_prec* p, int which, int level, int64_t* rp, int32_t* ci, double* v);
/* one V-cycle of component comp on level-0 input b */
int or_amg_vcycle(const or_prec* p, int which, int comp, const double* b, double* x);
// one level-0 smoother application on a scalar CSR matrix (kind 1 Chebyshev of degree count over
// [lambda_hat/ratio, lambda_hat] of D^{-1}A; kind 0 count l1-Jacobi sweeps); zero: start from x = 0
int or_smoother_apply(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* b, double* x,
                      int kind, int count, double ratio, int zero);
/* S_pp^(cpr-fs) (§5.3) as CSR, and the fixed-stress S_ff (§5.1) as 2x2 BSR */
int64_t or_spp_nnz(const or_prec* p);
int or_spp(const or_prec* p, int64_t* rp, int32_t* ci, double* v);
/* the (D_sp, D_pp) pairs added to the diagonal blocks of S_ff (2 per cell) */
int or_fs_diag(const or_prec* p, double* dfs);
/* ILU(0) inverse diagonal blocks inv(U_ii), 4 per cell */
int or_ilu_dinv(const or_prec* p, double* dinv);
/* apply M_L^{-1} (block ILU(0)) to a flow vector */
int or_ilu_apply(const or_prec* p, const double* w, double* dz);
/* option 1 of §5.3: `sweeps` sweeps of block Gauss-Seidel on the interleaved S_ff^(FS) from dz = 0, cells
   visited in red-black order (colour (i + j + k) mod 2, colour 0 first, ascending id within a colour) */
int or_gs_apply(const or_prec* p, const double* w, double* dz, int sweeps);

typedef struct {
  int32_t iters, restarts, converged, breakdown;
  double true_relres, est_relres;
} or_stats;

/* FGMRES(m) with right preconditioning (§4), x0 = 0 */
int or_fgmres(const or_system* s, or_prec* p, const double* b, double* x, double tol,
              int restart, int max_iters, or_stats* st);
/* Newton's method for one time step (§4 and its remarks on inexact Newton): the previous time level is the
   base state and the first iterate; each step solves J y = -R r by FGMRES under the two-stage preconditioner
   (mechanics hierarchy of the first step kept, §5.4) to the relative tolerance eta_k, with dx = C y
   (pressure in MPa) and backtracking; converged when ||R_0 r_k|| <= rtol ||R_0 r_0||. */
enum { OR_FORCING_FIXED = 0, OR_FORCING_EW = 1 };
typedef struct {
  double rtol;
  int32_t max_newton;
  int32_t forcing;         /* OR_FORCING_FIXED (eta_fixed) or OR_FORCING_EW (Eisenstat-Walker choice 2) */
  double eta_fixed;
  double ew_gamma, ew_omega, ew_eta0, ew_eta_max;
  int32_t max_backtracks;
  int32_t restart, max_linear;
} or_newton_params;
typedef struct {
  int32_t newton_iters, linear_iters, backtracks, converged;
  double rnorm[33];        /* ||R_0 r_k||, k = 0 .. newton_iters */
  double eta[32];
  int32_t lin_iters[32];
} or_newton_stats;
void or_newton_params_default(or_newton_params* np);
double or_ew_eta(const or_newton_params* np, int k, double rk, double rkm1, double eta_prev, double r0);
/* x_out: the converged x (u, then (s, p) per cell) relative to the base state */
int or_newton(const or_gen_params* gp, const or_prec_params* pp, const or_newton_params* np, double* x_out,
              or_newton_stats* st);

/* sequential fixed-stress strategy (§5.4 remark): Richardson iteration x <- x + M^{-1}(b - A x) from x0 = 0
   until ||b - A x|| <= tol ||b|| or max_iters applications of M^{-1} */
int or_richardson(const or_system* s, or_prec* p, const double* b, double* x, double tol, int max_iters,
                  or_stats* st);
/* the same Krylov loop on a diagonal operator with identity preconditioner */
int or_fgmres_diag(int64_t n, const double* diag, const double* b, double* x, double tol,
                   int restart, int max_iters, or_stats* st);

/* dense LU with partial pivoting of the whole Jacobian (n <= 6000) */
int or_dense_solve(const or_system* s, const double* b, double* x);
/* dense LU solve of a row-major n x n matrix (overwritten) */
int or_lu_solve(int64_t n, double* a, const double* b, double* x);

/* Terzaghi consolidation column (textbook closed form, not in the paper):
   nz cells of edge h, load sigma0 on top, drained top, rollers, fixed base.
   Writes cell pressures p[nsteps][nz] and times t[nsteps]; returns the
   undrained initial pressure in *p0 and the consolidation coefficient c_v. */
typedef struct {
  int32_t nz; double h; double E, nu, biot, kappa, mu, phi0, rho0, sigma0, dt;
  int32_t nsteps;
} or_terzaghi_params;
int or_terzaghi(const or_terzaghi_params* tp, double* t, double* p, double* p0, double* cv,
                double* newton_ratio);

#ifdef __cplusplus
}
#endif
#endif
