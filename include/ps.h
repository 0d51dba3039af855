/*
 * ps.h -- C ABI of the GB300 solver for one linearised fully-implicit
 * multiphase-poromechanics Jacobian (White, Castelletto, Klevtsov, Bui,
 * Osei-Kuffuor, Tchelepi, "A two-stage preconditioner for multiphase
 * poromechanics in reservoir simulation", arXiv 1812.05540).
 *
 * Problem (§4): solve A dx = b, A = [[A_uu, A_uf], [A_fu, A_ff]] (Eq. (jac_system)
 * regrouped as in §5.1), with right-preconditioned flexible GMRES under the
 * block-triangular preconditioner of §5.1 (Eq. (blk_tr_prec)) whose mechanics
 * stage is an AMG V-cycle on the separate-displacement-component block (§5.2)
 * and whose flow stage is the CPR two-stage operator of §5.3 (quasi-IMPES
 * pressure AMG followed by block ILU(0)), applied by Algorithm 1.  The solver
 * runs in two phases, setup then iterate, as §5.4 describes.
 *
 * Unknown ordering: x = [u (3 per node, node-major, components x,y,z);
 * f (2 per cell, interleaved (s, p))] -- the interleaved flow ordering of the
 * permutation P in §5.3.  Node id = i + (nx+1)(j + (ny+1)k), cell id =
 * i + nx(j + ny k), k = 0 at the bottom.
 *
 * Conventions for every entry point:
 *  - Pointers are device pointers unless ps_params.host_ptrs = 1 (then every
 *    array in ps_jacobian, rhs and x is a host pointer and the library copies).
 *  - The caller owns every pointer it passes; the library owns every handle.
 *  - All device work is enqueued on ps_params.stream (NULL = legacy stream);
 *    ps_setup and ps_solve synchronise that stream before returning.
 *  - Functions return ps_status and never abort; no device assert or trap is
 *    used.  The handle stays valid after PS_ERR_NOT_CONVERGED, PS_ERR_NAN and
 *    PS_ERR_TIMEOUT.  Not thread-safe per handle.
 */
#ifndef PS_H
#define PS_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PS_OK = 0,
  PS_ERR_INVALID = 1,        /* bad argument, shape or pattern */
  PS_ERR_OOM = 2,            /* device allocation failed */
  PS_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  PS_ERR_NOT_CONVERGED = 4,  /* max_iters reached; x holds the last iterate */
  PS_ERR_BREAKDOWN = 5,      /* Krylov breakdown before convergence */
  PS_ERR_NAN = 6,            /* NaN/Inf in the residual or the Hessenberg */
  PS_ERR_TIMEOUT = 7,        /* a bounded device wait gave up */
  PS_ERR_BUDGET = 8          /* the handle would exceed ps_params.hbm_budget */
} ps_status;

/* preconditioner precision: FP64; FP32 (FP64 Krylov, SpMV, fixed-stress diagonal and coarsest solve);
   or FP32 with the AMG prolongators and restrictors stored in BF16 (read as BF16, summed in FP32) */
enum { PS_FP64 = 0, PS_MIXED_FP32 = 1, PS_MIXED_BF16P = 2 };
enum { PS_SMOOTH_L1JACOBI = 0, PS_SMOOTH_CHEBYSHEV = 1 };
enum { PS_ILU_LEVEL_LAUNCH = 0, PS_ILU_PENCIL = 1 };
/* local stage M_L of §5.3: option 2, one sweep of block ILU(0) (default); option 1, local_sweeps sweeps of
   block Gauss-Seidel on the interleaved S_ff^(FS), cells taken in red-black order */
enum { PS_LOCAL_ILU0 = 0, PS_LOCAL_HBGS = 1 };
/* scope of the ILU(0) local stage: the whole flow system, or processor-local (§6: each process factors
   the rows it owns), with subdomains of PS_ILU_TILE_Y x PS_ILU_TILE_Z cell columns in (y, z) spanning x */
enum { PS_ILU_GLOBAL = 0, PS_ILU_LOCAL = 1 };
/* mechanics AMG M_uu: on the separate-displacement-component approximation A_uu^(SDC) (§5.2, default), or
   rigid-body-mode smoothed aggregation on the full A_uu (the usual elasticity AMG the paper sets aside) */
enum { PS_MECH_SDC = 0, PS_MECH_RBM = 1 };
#define PS_ILU_TILE_Y 16
#define PS_ILU_TILE_Z 8
/* CPR pressure reduction of §5.3: quasi-IMPES (diagonal entries of A_ss, A_ps; default) or true-IMPES
   (column sums of A_ss, A_ps) */
enum { PS_CPR_QUASI_IMPES = 0, PS_CPR_TRUE_IMPES = 1 };
/* outer iteration: flexible GMRES (default), or the sequential fixed-stress strategy of the §5.4 remark,
   the preconditioner inside a Richardson iteration x <- x + M^{-1}(b - A x) (one mechanics-then-flow pass
   per iteration; max_iters bounds the passes) */
enum { PS_SOLVER_FGMRES = 0, PS_SOLVER_RICHARDSON = 1 };
/* fixed-stress diagonal (D_sp, D_pp) added to A_ff: the caller's d_fs (default), or the row-sum lumping of
   the §5.1 remark, -diag(A_su w) and -diag(A_pu w) with w = M_uu^{-1} (A_up e) (one FP64 mechanics
   V-cycle per displacement component; d_fs is then ignored) */
enum { PS_FS_GIVEN = 0, PS_FS_RSL = 1 };
enum { PS_ORTHO_MGS = 0, PS_ORTHO_CGS2 = 1 };    /* Arnoldi orthogonalisation */

/* Cartesian box of nx*ny*nz cubic cells (§6 grids); hx = hy = hz. */
typedef struct {
  int32_t nx, ny, nz;
  double hx, hy, hz;
} ps_grid;

/* Block-sparse row matrix: n_brow block rows of br x bc row-major FP64 blocks,
   column indices sorted ascending within each row. */
typedef struct {
  int64_t n_brow, n_bcol, nnzb;
  int32_t br, bc;
  const int64_t* rowptr; /* n_brow + 1 */
  const int32_t* colind; /* nnzb */
  const double* val;     /* nnzb * br * bc */
} ps_bsr;

/* Jacobian blocks of §5.1 (App. B expressions):
   A_uu: 3x3, node x node, Q1 27-point pattern;
   A_uf: 3x2, node x cell, columns (s, p) = [A_us A_up];
   A_fu: 2x3, cell x node, rows (s, p) = [A_su; A_pu];
   A_ff: 2x2, cell x cell, TPFA 7-point pattern, [[A_ss A_sp] [A_ps A_pp]]. */
typedef struct {
  ps_bsr A_uu, A_uf, A_fu, A_ff;
  const double* d_fs;         /* 2 per cell: fixed-stress (D_sp, D_pp) of §5.1, scaled like A_ff */
  const uint8_t* dirichlet_u; /* 3 per node, 1 = constrained (identity row); may be NULL */
} ps_jacobian;

typedef struct {
  int32_t precision;          /* PS_FP64, PS_MIXED_FP32 (FP32 preconditioner, FP64 Krylov) or PS_MIXED_BF16P */
  int32_t restart;            /* FGMRES restart length m (default 100) */
  int32_t max_iters;          /* total Krylov iterations (default 1000) */
  int32_t smoother;           /* PS_SMOOTH_* (default Chebyshev) */
  int32_t pre, post;          /* l1-Jacobi sweeps (default 1, 1) */
  int32_t cheb_degree;        /* Chebyshev degree (default 2) */
  double cheb_ratio;          /* Chebyshev interval [lambda/ratio, lambda] (default 20) */
  double theta_u, theta_p;    /* strength thresholds at level 0, halved per level (0.08) */
  int32_t coarse_max_u;       /* coarsest mechanics level size in nodes (500) */
  int32_t coarse_max_p;       /* coarsest pressure level size in cells (500) */
  int32_t max_levels;         /* (25) */
  int32_t ilu_mode;           /* PS_ILU_PENCIL (default: sync-free wavefront) or PS_ILU_LEVEL_LAUNCH */
  int64_t spin_limit;         /* polls of a wavefront wait before PS_ERR_TIMEOUT (default 2e6, ~1 s) */
  int32_t host_ptrs;          /* 1: jacobian arrays, rhs and x are host pointers */
  int64_t hbm_budget;         /* bytes the handle may hold; 0 = unlimited */
  void* stream;               /* cudaStream_t */
  int32_t test_stall_wave;    /* testing only, 0 = off: k > 0 makes wavefront CTA k-1 skip its
                                 work so that the bounded waits of its consumers run out and
                                 ps_solve returns PS_ERR_TIMEOUT (no fault, no hang) */
  int32_t ortho;              /* PS_ORTHO_MGS (default: modified Gram-Schmidt, one cooperative launch
                                 per Arnoldi step) or PS_ORTHO_CGS2 (classical Gram-Schmidt with the
                                 DGKS reorthogonalisation test) */
  int32_t test_stall_gs;      /* testing only, 0 = off: k > 0 makes CTA k-1 of the Gram-Schmidt
                                 launch skip its work, so the grid barrier waits of the others run
                                 out and ps_solve returns PS_ERR_TIMEOUT (no fault, no hang) */
  int32_t ortho_sweep;        /* PS_ORTHO_MGS: basis vectors projected out per sweep over the rows
                                 (1, 2, 4 or 8; default 8).  The coefficients equal those of
                                 one-vector-at-a-time modified Gram-Schmidt in exact arithmetic
                                 (forward substitution with the in-block Gram entries); larger
                                 sweeps need fewer grid barriers */
  int32_t local_stage;        /* PS_LOCAL_ILU0 (default) or PS_LOCAL_HBGS (§5.3 option 1) */
  int32_t local_sweeps;       /* PS_LOCAL_HBGS: block Gauss-Seidel sweeps (default 3, as in §6.1) */
  int32_t cpr_reduction;      /* PS_CPR_QUASI_IMPES (default) or PS_CPR_TRUE_IMPES */
  int32_t solver;             /* PS_SOLVER_FGMRES (default) or PS_SOLVER_RICHARDSON */
  int32_t fs_mode;            /* PS_FS_GIVEN (default) or PS_FS_RSL */
  int32_t vcycle_tail;        /* 0 (default): one kernel per V-cycle step, replayed as a CUDA graph;
                                 1: the levels below the finest as one cooperative launch with bounded grid
                                 barriers between their steps; 2: the levels from the first one of at most
                                 1024 rows as one launch of a 16-CTA thread-block cluster with hardware cluster
                                 barriers (both: Chebyshev degree 2, FP32/FP64 transfer operators).  Same
                                 results every way; other values PS_ERR_INVALID. */
  int32_t pdl;                /* 1 (default): each V-cycle kernel after the first is launched with
                                 programmatic dependent launch, so its CTAs are scheduled while the
                                 previous kernel drains and wait on the device for its completion;
                                 0: plain stream order.  Same results either way. */
  int32_t ilu_scope;          /* PS_ILU_LOCAL (default): processor-local ILU(0) as in the paper's runs, the
                                 ILU(0) of S_ff^(FS) without the blocks that couple different subdomains
                                 (columns of PS_ILU_TILE_Y x PS_ILU_TILE_Z cells), whose sweeps need no
                                 exchange between subdomains; PS_ILU_GLOBAL: ILU(0) of the whole
                                 S_ff^(FS), the sweeps exchanging tile faces through tagged halo words */
  int32_t mech_amg;           /* PS_MECH_SDC (default) or PS_MECH_RBM: 3 x 3 blocks on the nodes, the six
                                 rigid-body modes as near-nullspace, 6 x 6 blocks on the aggregates below,
                                 QR-based tentative prolongator, Jacobi-smoothed P, Galerkin levels;
                                 Chebyshev smoothing only (PS_ERR_INVALID otherwise) */
  int32_t autotune;           /* 1: at setup, time the CSR row kernels of every coarse level (operator, P, R)
                                 with half, the same and twice the lanes per row that the mean row length
                                 gives, and keep the fastest (within 3 %% the default stays); choices are cached
                                 per process by level shape, so equal hierarchies get equal schedules.  The
                                 lanes change only the order of a row's FP32/FP64 sums.  0 (default): lanes
                                 from the mean row length alone. */
} ps_params;

typedef struct {
  int32_t iters, restarts;
  double true_relres, est_relres;  /* ||b - A x|| / ||b|| in FP64, Arnoldi estimate */
  float ms_setup_u, ms_setup_f, ms_solve;
  int64_t bytes_model;              /* algorithmic HBM bytes of the solve */
  int64_t handle_bytes;             /* device bytes held by the handle */
  int32_t levels_u, levels_p;
  float ms_prec, ms_spmv, ms_orth;  /* solve time in Algorithm 1, the Jacobian SpMV and Gram-Schmidt */
  int32_t reorth;                   /* Arnoldi steps that needed the second Gram-Schmidt pass */
  float ms_vcycle_u, ms_flow24, ms_vcycle_p, ms_ilu;  /* parts of ms_prec: Algorithm 1 step 1, steps
                                                          2-4, step 5, steps 6-8 */
  float ms_copy_in;                 /* part of ms_setup_u: copying the four Jacobian blocks and d_fs into
                                       the handle (host to device with host_ptrs = 1) */
} ps_stats;

typedef struct ps_handle ps_handle;

/* Fill *p with the defaults listed above. */
void ps_params_default(ps_params* p);

/* Setup phase of §5.4: validates shapes (A_uu rows = nodes, A_ff rows = cells of
   *grid, 7-point A_ff pattern), copies the FP64 blocks, builds S_ff^(FS) (§5.1),
   the quasi-IMPES S_pp (§5.3), the mechanics AMG on A_uu^(SDC) (§5.2), the
   pressure AMG on S_pp, block ILU(0) of S_ff^(FS) and the Krylov workspace.
   On success *out owns all of it until ps_free.  Errors: PS_ERR_INVALID,
   PS_ERR_OOM, PS_ERR_BUDGET, PS_ERR_CUDA. */
ps_status ps_setup(const ps_jacobian* jac, const ps_grid* grid, const ps_params* params,
                   ps_handle** out);

/* Per-Newton flow setup of §5.4: new A_fu, A_ff and d_fs values (patterns as
   given to ps_setup) rebuild the flow stage (S_ff^(FS), S_pp, pressure AMG,
   local stage) while the mechanics AMG built by ps_setup is kept.  When
   jac->A_uu.val and jac->A_uf.val are non-NULL their new values (same
   patterns) replace the stored ones for the outer Jacobian SpMV; NULL keeps
   the stored values.  The stored Jacobian then is the new one throughout,
   so ps_solve solves the new system.  A row-sum-lumped fixed-stress diagonal
   (PS_FS_RSL) keeps the M_uu^{-1} A_up e vector of ps_setup and applies the
   new A_fu to it.  Errors: PS_ERR_INVALID (shape or pattern change). */
ps_status ps_setup_flow(ps_handle* h, const ps_jacobian* jac);

/* Testing only: set ps_params.test_stall_wave on an existing handle (0 = off). */
ps_status ps_set_test_stall(ps_handle* h, int32_t wave_cta_plus_one);

/* Testing only: set ps_params.test_stall_gs on an existing handle (0 = off). */
ps_status ps_set_test_stall_gs(ps_handle* h, int32_t cta_plus_one);

/* Iteration phase: x = FGMRES(A, M^{-1}, rhs) from x0 = 0 to the true FP64
   relative residual tol.  rhs, x: n = 3*nodes + 2*cells doubles.
   PS_ERR_NOT_CONVERGED still fills x and *st (st may be NULL). */
ps_status ps_solve(ps_handle* h, const double* rhs, double* x, double tol, ps_stats* st);

/* Batched setup: n independent systems (jac[i] on grid[i]), each with params except the stream: handle i
   gets a stream of its own (created by the library and destroyed by ps_free).  The setups run on up to
   eight host threads at once, so their kernels overlap on the device.  On failure every handle made so
   far is freed, out[] is zeroed and the first failing status is returned.  The paper solves one system
   at a time (§5.4); this is the batching layer around that setup. */
ps_status ps_setup_batch(int32_t n, const ps_jacobian* jac, const ps_grid* grid, const ps_params* params,
                         ps_handle** out);

/* Batched iteration phase: the FGMRES solves of n handles (rhs[i], x[i] as in ps_solve).  The systems
   are dealt round-robin to up to eight host threads; each thread advances its group in lockstep, one
   Arnoldi step (or cycle end) of every unfinished system per round, each on its handle's stream, with
   one host synchronisation per round for the group.  Each system runs the kernels of ps_solve in the
   same order, so x[i] equals what ps_solve gives for it.  stats[i] (may be NULL) gets each system's
   statistics; the first non-OK status in system order is returned.  Handles with the Richardson solver
   are solved whole by their group's thread.  Handles must be distinct. */
ps_status ps_solve_batch(int32_t n, ps_handle* const* h, const double* const* rhs, double* const* x, double tol,
                         ps_stats* stats);

/* y = A x with the stored FP64 Jacobian (device pointers). */
ps_status ps_spmv(ps_handle* h, const double* x, double* y);

/* z = M^{-1} v, Algorithm 1 (device pointers, FP64 in and out). */
ps_status ps_apply_prec(ps_handle* h, const double* v, double* z);

/* Hierarchy inspection for parity checks: which = 0 mechanics, 1 pressure.
   Returns the level count; level_n/level_nnz/agg are copied to host memory. */
int32_t ps_amg_nlevels(ps_handle* h, int32_t which);
ps_status ps_amg_level_info(ps_handle* h, int32_t which, int32_t level, int64_t* n, int64_t* nnz,
                            int64_t* nagg);
/* Shape of one level as the V-cycle applies it (for traffic accounting): shape[0] rows, [1] operator
   entries, [2] rows of the next level (0 on the coarsest), [3] prolongator entries (R = P^T has as
   many), [4] stencil slots of the level's stencil copy (27 or 7; 0 when the level runs in CSR form),
   [5] bytes per stored operator value in the apply precision (4 or 8), [6] bytes per stored P and R
   value (2 with BF16 transfer operators), [7] 1 on the coarsest level (dense FP64 inverse). */
ps_status ps_amg_level_shape(ps_handle* h, int32_t which, int32_t level, int64_t* shape);
/* host copies: rowptr[n+1], colind[nnz], val[nnz*ncomp] (ncomp 3 or 1), agg[n] (-1 excluded) */
ps_status ps_amg_level_copy(ps_handle* h, int32_t which, int32_t level, int64_t* rowptr, int32_t* colind,
                            double* val, int32_t* agg);
/* Rigid-body-mode hierarchy (mech_amg = PS_MECH_RBM) for parity checks: the level count (0 otherwise);
   shape[0] block rows, [1] block size b (3 on the finest level, 6 below), [2] operator blocks,
   [3] aggregates (0 on the coarsest level), [4] prolongator blocks, [5] 1 on the coarsest level; host
   copies of a level's operator (rowptr[n+1], colind[nnzb], val[nnzb*b*b] row-major blocks) and aggregates
   agg[n], and of its prolongator (b x 6 blocks) */
int32_t ps_rbm_nlevels(ps_handle* h);
ps_status ps_rbm_level_shape(ps_handle* h, int32_t level, int64_t* shape);
ps_status ps_rbm_level_copy(ps_handle* h, int32_t level, int64_t* rowptr, int32_t* colind, double* val,
                            int32_t* agg);
ps_status ps_rbm_prolongator_copy(ps_handle* h, int32_t level, int64_t* rowptr, int32_t* colind, double* val);
/* S_pp values in the A_ff pattern and ILU inverse diagonal blocks (host copies) */
ps_status ps_flow_copy(ps_handle* h, double* spp, double* dinv);

/* Residual without device allocation: r = b - A x and *rnorm2 = ||r||^2 for
   the FP64 Jacobian blocks in *jac (device pointers, int64 row pointers as in
   ps_bsr), x, b, r of length n and rnorm2 (one double) device pointers.  The
   paper has no counterpart: this entry point exists for callers that manage
   all device memory themselves (for instance a simulator that reserves its HBM
   at start-up so a long run cannot fail on an allocation, or a process whose
   allocator is capped) and so cannot let the library call cudaMalloc.  It
   allocates nothing: its only scratch (the partial sums of ||r||^2) is a fixed
   static device array of (2^19 + 1024) doubles, 4 MiB, which every GPU that
   loads the library holds until exit.  The first call on each device looks up
   that array's device address (cudaGetSymbolAddress) with the device current;
   make that first call before any stream capture.  The address is kept for the
   life of the process: do not call this entry point after cudaDeviceReset.
   The partial sums fill one slot per 8 rows of each block, so a system is
   accepted when ceil(nodes / 8) + ceil(cells / 8) <= 2^19 (about 2^22 rows in
   total); larger ones are rejected with PS_ERR_INVALID.  r must not overlap x
   or b (r == x or r == b is rejected with PS_ERR_INVALID).  Every call shares
   the array, so calls that overlap on the GPU race: the caller must not run two
   at once.  Work is enqueued on stream (NULL = legacy stream) and not
   synchronised; *rnorm2 is valid once the stream reaches that point. */
ps_status ps_residual_noalloc(const ps_jacobian* jac, const ps_grid* grid, const double* x, const double* b,
                              double* r, double* rnorm2, void* stream);

/* Frees everything the handle owns (synchronises its stream). */
void ps_free(ps_handle* h);

/* ---- request server: many independent solves in flight (batched and served workloads) ----
   A server runs whole requests -- ps_setup, one ps_solve per right-hand side, ps_free -- on `slots`
   worker threads, each with its own CUDA stream, so requests overlap on the device.  Requests are
   admitted first come, first served when a worker is idle and the estimated device bytes of the
   request's handle (ps_setup_bytes_estimate) fit under hbm_budget next to the requests in flight.
   The paper solves one system at a time (§5.4); this is the batching/serving layer around that
   solve, with the same kernels, so a request gives the same x alone and in the mix. */
typedef struct ps_server ps_server;
typedef struct {
  int32_t slots;          /* requests in flight at once (worker threads / CUDA streams), 1..256 */
  int64_t hbm_budget;     /* bytes of handles in flight at once, by estimate; 0 = unlimited */
  ps_params params;       /* solver parameters of every request (params.stream is ignored) */
} ps_server_params;
typedef struct {
  uint64_t ticket;
  ps_status status;                  /* first failing status of the request's setup or solves */
  int32_t nrhs, iters;               /* iterations summed over the right-hand sides */
  double worst_relres;               /* largest true FP64 relative residual over the right-hand sides */
  double t_arrival, t_start, t_end;  /* seconds on the server clock (ps_server_clock) */
  int64_t bytes;                     /* device bytes the request's handle held */
} ps_request_info;
typedef struct {
  int64_t submitted, completed;
  int64_t max_inflight_bytes;        /* largest sum of admitted estimates seen */
  int64_t max_inflight_requests;
} ps_server_info;

/* Device bytes a handle for this Jacobian will hold (estimate with a 20 % margin).  Host arithmetic on
   the block counts and the grid only: the array pointers in jac are not read and no device is used.
   Counts the Jacobian copies, the FP64 stencil copy, both AMG hierarchies, the flow stage with its
   ILU(0) sweep records, the Krylov bases and the work vectors.  Returns 0 when an argument is NULL. */
int64_t ps_setup_bytes_estimate(const ps_jacobian* jac, const ps_grid* grid, const ps_params* params);
/* Starts the worker threads on the current device.  Errors: PS_ERR_INVALID. */
ps_status ps_server_create(const ps_server_params* params, ps_server** out);
/* Seconds since ps_server_create (steady clock). */
double ps_server_clock(const ps_server* s);
/* Queues one request: nrhs right-hand sides rhs[k] and solutions x[k] (device pointers, or host pointers
   with params.host_ptrs = 1), relative tolerance tol; t_arrival (server clock, < 0 = now) is the
   arrival time its latency is measured from.  The caller keeps every array of *jac, rhs[k] and x[k]
   alive and untouched until ps_server_wait returns for the ticket.  Errors: PS_ERR_INVALID,
   PS_ERR_BUDGET (estimate above hbm_budget; nothing queued). */
ps_status ps_server_submit(ps_server* s, const ps_jacobian* jac, const ps_grid* grid, int32_t nrhs,
                           const double* const* rhs, double* const* x, double tol, double t_arrival,
                           uint64_t* ticket);
/* Blocks until the request is done, fills *info (may be NULL) and returns its status; the ticket is
   then forgotten. */
ps_status ps_server_wait(ps_server* s, uint64_t ticket, ps_request_info* info);
ps_status ps_server_info_get(ps_server* s, ps_server_info* info);
/* Runs every queued request to completion, then stops the workers and frees the server. */
void ps_server_destroy(ps_server* s);

/* ---- seeded synthetic Jacobian generator (test input; §6 physics) ---- */
enum { PS_FIELDS_LOGNORMAL = 0, PS_FIELDS_LAYERED = 1, PS_FIELDS_CHANNELS = 2,
       PS_FIELDS_HOMOGENEOUS = 3 };
enum {
  PS_GEN_GRAVITY = 1 << 0, PS_GEN_DIRICHLET = 1 << 1, PS_GEN_SCALE = 1 << 2,
  PS_GEN_ACCUM = 1 << 3, PS_GEN_FLUX = 1 << 4, PS_GEN_FLUX_SAT = 1 << 5,
  PS_GEN_COUPLING = 1 << 6, PS_GEN_ALL = 0x7f,
  /* option, not in PS_GEN_ALL: Peaceman wells under bottom-hole pressure control (§3 well model, Table 1): a
     water injector in the cell column (0, 0) and a producer in (nx-1, ny-1), both perforating every layer,
     bottom-hole pressures 5 MPa above and below the hydrostatic formation pressure at the top perforation,
     built up linearly over one day (a step of dt reaches the fraction min(dt / 1 day, 1)) */
  PS_GEN_WELLS = 1 << 7
};

typedef struct {
  int32_t nx, ny, nz;
  double h;
  uint64_t seed;
  int32_t field_kind;
  uint32_t flags;
  double dt, biot, c_w, c_nw, c_r, mu_w, mu_nw, rho_w0, rho_nw0, rho_s0, s_wr, s_nwr, grav, p_ref, dp_amp, corey;
  double E0, nu0, kappa0, phi0, sw0;
  int32_t fs_modulus;  /* fixed-stress diagonal of §5.1 with the drained bulk modulus K_dr (0, default) or
                          the uniaxial modulus K_dr + 4G/3 (1; the §5.1 remark on one-dimensional loading) */
} ps_gen_params;

/* A generated system: every pointer is device memory owned by the library. */
typedef struct {
  ps_jacobian jac;
  ps_grid grid;
  double* rhs;
  int64_t n_nodes, n_cells, n_u, n_f, n;
  double alpha_u, alpha_f;        /* row scales of §4 (remark on block-row scaling) */
  double *E, *nu, *kh, *kv, *phi0, *sw, *p;  /* cell fields at the linearisation point */
} ps_system;

/* Defaults of the synthetic configurations (0: 8x8x4 lognormal, 1: 64x64x32
   layered, 2: 60x220x85 channelised, 3: 16x16x8 layered). */
void ps_gen_default(ps_gen_params* gp, int32_t config);
/* Generates the Jacobian, d_fs and a seeded rhs on the device (stream may be
   NULL).  *out is owned by the library until ps_system_free. */
ps_status ps_generate(const ps_gen_params* gp, void* stream, ps_system** out);
void ps_system_free(ps_system* s);

/* ---- the generated problem away from its linearisation point: Newton's method for one time step ----
   The previous time level is the generator's base state (zero displacement, the saturation and pressure
   fields sw and p) and x holds the unknowns relative to it (u; then (s, p) per cell; pressure in Pa).

   ps_assemble_at: re-assembles sys's Jacobian values (App. B blocks, d_fs, Dirichlet elimination, scaling
   with alpha_u, alpha_f recomputed, as ps_generate does at the base state) at base + dx, and writes the
   unscaled residual of the discrete equations (§3 weak form and TPFA balances, App. B) there into r,
   Dirichlet rows zero.  The porosity of the Jacobian's blocks uses the element-mean volumetric strain, the
   residual the strain at each Gauss point.  dx, r: device arrays of sys->n doubles (r may be NULL); sys must
   come from ps_generate(gp); the rhs and patterns are kept.  ps_residual_at: the residual alone. */
ps_status ps_assemble_at(const ps_gen_params* gp, ps_system* sys, const double* dx, double* r, void* stream);
ps_status ps_residual_at(const ps_gen_params* gp, ps_system* sys, const double* dx, double* r, void* stream);

/* Newton's method (§4 and its remarks on inexact Newton): x_0 = 0; step k solves J_k y = -R_k r_k (R_k the
   rows' scaling of J_k) by ps_solve under lin's preconditioner to the relative tolerance eta_k, keeping the
   mechanics hierarchy of the first step (§5.4: ps_setup once, then ps_setup_flow), and sets
   x_{k+1} = x_k + lambda C y (C: pressure unknowns from MPa to Pa), halving lambda up to max_backtracks times
   while ||R_0 r|| > (1 - 1e-4 lambda) ||R_0 r_k||.  Converged when ||R_0 r_k|| <= rtol ||R_0 r_0||, R_0 the
   base state's row scaling.  eta_k: eta_fixed (PS_FORCING_FIXED, the paper's runs use 1e-6) or Eisenstat
   and Walker's choice gamma (||r_k|| / ||r_{k-1}||)^omega, eta_0 = ew_eta0, with the paper's safeguard
   max(eta_k, gamma eta_{k-1}^omega) when gamma eta_{k-1}^omega > 0.1, capped at ew_eta_max and kept at or
   above 0.5 rtol ||r_0|| / ||r_k|| (PS_FORCING_EW).  x: device array of n doubles (the final iterate). */
enum { PS_FORCING_FIXED = 0, PS_FORCING_EW = 1 };
typedef struct {
  double rtol;              /* default 1e-5 (the paper's Newton tolerance, Table 1) */
  int32_t max_newton;       /* default 12 (at most 32) */
  int32_t forcing;          /* PS_FORCING_EW (default) or PS_FORCING_FIXED */
  double eta_fixed;         /* default 1e-6 */
  double ew_gamma, ew_omega, ew_eta0, ew_eta_max;  /* defaults 0.9, 2, 0.1 (the paper's values), 0.1 */
  int32_t max_backtracks;   /* default 4 */
} ps_newton_params;
typedef struct {
  int32_t newton_iters, linear_iters, backtracks, converged;
  double rnorm[33];         /* ||R_0 r_k||, k = 0 .. newton_iters */
  double eta[32];           /* Krylov tolerance of each step */
  int32_t lin_iters[32];    /* FGMRES iterations of each step */
  float ms_assemble, ms_linear, ms_total;  /* assembly (Jacobian and residuals), setup + solve, wall time */
} ps_newton_stats;
void ps_newton_params_default(ps_newton_params* np);
/* eta_k of the rule above (k, ||r_k||, ||r_{k-1}||, eta_{k-1}, ||r_0||) */
double ps_newton_eta(const ps_newton_params* np, int32_t k, double rk, double rkm1, double eta_prev, double r0);
/* PS_ERR_NOT_CONVERGED when max_newton steps did not reach rtol (x and stats still filled) */
ps_status ps_newton(const ps_gen_params* gp, const ps_params* lin, const ps_newton_params* np, double* x,
                    ps_newton_stats* stats);

const char* ps_strerror(ps_status s);

/* Number of CUDA kernels this library has launched in the process so far
   (monotone counter; differences bracket a region of interest). */
int64_t ps_launch_count(void);

/* Number of device allocations the library has made in the process so far (monotone counter; every
   device buffer of a handle, generator output or server request is one). */
int64_t ps_alloc_count(void);

/* Device bytes the library's memory pool on the current device holds (*reserved, including freed blocks it
   keeps for reuse) and has handed out (*used). */
ps_status ps_pool_bytes(int64_t* reserved, int64_t* used);

#ifdef __cplusplus
}
#endif
#endif
