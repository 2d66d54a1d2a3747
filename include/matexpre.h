/*
 * matexpre.h -- C ABI of the GB300 (sm_103a) MatExPre library.
 *
 * MatExPre (arXiv 2506.03617) preconditions the finite-difference Helmholtz
 * operator with PML and complex shift through matrix-exponential actions:
 * Algorithm 1 computes r <- psi_1(i t A_s) r and then solves
 * (I - exp(i t A_s)) w = r with GMRES to a relative tolerance fprtol; outer
 * flexible GMRES uses w as the preconditioned direction (Sec. 3.4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  Layout.  A grid vector is complex128, interleaved (re, im), one value per
 *    unknown, x fastest: index = i + n_x (j + n_y k).  Axis d holds
 *    n_d = N_d + 2 npml unknowns; unknown j sits at x_j = (j - npml + 1/2) h and
 *    the Dirichlet zero values sit at j = -1 and j = n_d.
 *  Memory.  Unless a name ends in _host, vector arguments are DEVICE pointers
 *    on the problem's device, 16-byte aligned, owned by the caller, and must
 *    not alias each other.  The library owns the medium copy, the PML profiles
 *    and the Krylov workspace; all are released by mxp_destroy.
 *  Streams.  All work is enqueued on the stream given to mxp_create (NULL = the
 *    legacy default stream).  Calls that return statistics or decide on
 *    convergence synchronise that stream.
 *  Errors.  Every call returns an mxp_status; no exception crosses the ABI.
 *    On failure mxp_last_error() returns a thread-local message.  Invalid
 *    arguments are rejected before any device work is enqueued.
 *  Threads.  A problem handle may be used by one host thread at a time.
 */
#ifndef MATEXPRE_H
#define MATEXPRE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MXP_OK = 0,
    MXP_EINVAL = 1,       /* invalid argument (sizes, NULL, non-finite values) */
    MXP_ENOMEM = 2,       /* device or host allocation failed */
    MXP_ECUDA = 3,        /* a CUDA runtime call failed */
    MXP_ENOCONV = 4,      /* iteration limit reached before the tolerance */
    MXP_EBREAKDOWN = 5,   /* reserved: the solvers stop at h_{j+1,j} = 0 (a lucky breakdown) and never return it */
    MXP_ENAN = 6,         /* NaN or Inf met in a residual */
    MXP_ETIMEOUT = 7      /* a bounded device-side wait gave up */
} mxp_status;

/* Precision of the matrix-exponential actions inside the MatExPre apply.
 * The Krylov bases, dot products, Hessenberg/Givens algebra of both GMRES
 * levels and every residual check stay complex128/FP64 in all modes. */
typedef enum {
    MXP_C128 = 0,         /* complex128 storage and arithmetic */
    MXP_C64 = 1,          /* complex64 storage and arithmetic */
    MXP_BF16S = 2         /* bfloat16 storage of the recurrence vectors and
                             float storage of the medium, float arithmetic */
} mxp_precision;

/* Grid: dim = 2 or 3; n_interior[d] = N_d interior cells (>= 1) for d < dim;
 * npml = PML cells on each side (>= 0); h = mesh size (> 0), normally
 * 1 / max_d N_d (the paper scales the largest interior extent to 1, Sec. 4). */
typedef struct {
    int dim;
    int64_t n_interior[3];
    int npml;
    double h;
} mxp_grid;

/* Method parameters (Sec. 3.3-3.4, Sec. 4).
 *  omega      angular frequency (> 0)
 *  c_pml      PML strength C_pml of Eq. pml-1d-s (>= 0; paper: 20)
 *  shift_s    complex shift s of A_s = A + i omega^2 s diag(1/c^2) (>= 0)
 *  t          time length of the exponential integrators (> 0)
 *  fprtol     inner GMRES relative tolerance of Algorithm 1 (0 < fprtol < 1)
 *  exp_tol    truncation tolerance of each exp / psi_1 action (0 < exp_tol < 1)
 *  inner_restart  inner GMRES restart length (1 .. 64)
 *  inner_maxit    cap on inner iterations per apply (>= 1)
 *  inner_fixed    if > 0: exactly this many inner iterations, tolerance
 *                 ignored (makes the apply a fixed linear map)
 *  prec       precision of the exp / psi_1 actions
 *  theta_max  largest sub-step norm ||t A_s'||/S used by the Taylor actions
 *             (0 = default: 6 for MXP_C128, 4 otherwise)
 *  fuse_k     Taylor steps fused per pass by the tiled 2D kernels of the
 *             low-precision modes: 0 = chosen by the autotuner, 1 = unfused,
 *             K > 1 = only tile shapes fusing K steps
 *  tile_cfg   -1 = autotune the tile shape; >= 0 forces that fused tile
 *             configuration (2D, MXP_C64 / MXP_BF16S only; see
 *             mxp_num_tile_configs)
 *  persist_cfg  persistent exp-action kernel (2D, MXP_C64 / MXP_BF16S): one
 *             cooperative launch per exp action with the grid held on chip;
 *             -1 = used when the autotuner finds it faster, -2 = never,
 *             0 .. mxp_num_persist_configs() - 1 = force that configuration when
 *             the grid fits the GPU and, for a problem with sound-hard / absorbing
 *             faces, the configuration adds face terms (otherwise the per-point
 *             sweep is used)
 *  precond    preconditioner of mxp_apply_matexpre and mxp_solve: 0 = Algorithm 1
 *             (default); 1 = the truncated Neumann series of Sec. 3.2,
 *             P_N r = (sum_{n=0}^{N} exp(i t A_s)^n) psi_1(i t A_s) r (constant -i t
 *             dropped; a fixed linear map, no inner GMRES; Thm. 3.1); 2 = Algorithm 1's
 *             steps on the second inverse formula of Sec. 3.1,
 *             A^{-1} = -i t (I - psi_1(i t A))^{-1} psi_2(i t A): r~ = psi_2(i t A_s) r
 *             and GMRES on (I - psi_1(i t A_s)) w = r~ to fprtol (w ~ (i/t) A_s^{-1} r)
 *  neumann_n  N of P_N (>= 0) */
typedef struct {
    double omega, c_pml, shift_s, t, fprtol, exp_tol;
    int inner_restart, inner_maxit, inner_fixed;
    mxp_precision prec;
    double theta_max;
    int fuse_k;
    int tile_cfg;
    int persist_cfg;
    int precond;
    int neumann_n;
} mxp_params;

/* Statistics of one MatExPre apply (Algorithm 1). */
typedef struct {
    int inner_iters;          /* inner GMRES iterations */
    int converged;            /* inner tolerance met (1) or not (0) */
    double inner_relres;      /* final inner residual estimate / ||psi_1 r|| */
    int64_t stencil_passes;   /* Taylor steps (stencil sweeps) executed */
    int64_t pt_updates;       /* stencil_passes * unknowns */
} mxp_apply_stats;

/* Outer solve options.  rtol: stop when ||b - A x|| <= rtol ||b|| (true
 * residual, unshifted A); restart: FGMRES restart (1 .. 64); maxit: cap on
 * outer iterations; x0_given: nonzero = x holds the initial guess on entry,
 * zero = start from x = 0. */
typedef struct {
    double rtol;
    int restart;
    int maxit;
    int x0_given;
} mxp_solve_opts;

typedef struct {
    int outer_iters;
    int inner_iters_total;
    int converged;
    double true_relres;        /* ||b - A x|| / ||b|| at return */
    double est_relres;         /* last FGMRES estimate / ||b|| */
    int64_t stencil_passes;    /* all stencil sweeps (actions + operator) */
    int64_t pt_updates;        /* sum over sweeps of the unknowns touched */
    double seconds;            /* wall time of the call (host clock) */
    int nn_accepted;           /* learned-stage directions kept (mxp_attach_cnn) */
    int nn_rejected;           /* learned-stage directions replaced by MatExPre */
} mxp_solve_stats;

typedef struct mxp_problem mxp_problem;   /* opaque, library-owned */

/* Create a problem on `device` with wave speed c_host (host array of
 * prod_d n_d doubles, x fastest, every value finite and > 0).  Parameters
 * start at the paper defaults for ppw 10 w.r.t. min c (mxp_default_params).
 * `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 * Follows the problem statement of Eq. helmholtz and Eq. pml-1d-s. */
mxp_status mxp_create(const mxp_grid *grid, const double *c_host, int device,
                      void *cuda_stream, mxp_problem **out);

/* Create a problem on a slab of a larger grid: rows [row0, row0 + nrows) of the
 * last axis of `grid` (the y rows in 2D, the z planes in 3D), for a slab
 * decomposition of one grid over several GPUs (the MPI / DMDA scheme of Sec. 4
 * with one slab per rank and halo rows exchanged between ranks).  c_slab_host
 * holds the wave speed of those rows (x fastest); c_range = {min, max} of c over
 * the whole grid.  The PML coefficients follow the rows' global positions and
 * the shift and Taylor plan are those of the whole grid (every slab of a grid
 * gets the same mu, S and m), so that steps on overlapping slabs agree.  Beyond
 * the slab's first and last rows the operator sees zero values: a caller keeps
 * the rows it owns exact by running K steps on its rows plus K halo rows on each
 * side, then exchanging halos.  Slabs run through mxp_horner_step and
 * mxp_apply_operator (complex128); the whole-grid entry points (actions,
 * MatExPre, solves, boundary faces, the learned stage) return MXP_EINVAL for a
 * slab.  MXP_EINVAL also for rows outside the grid or a range that does not
 * contain the slab's speeds. */
mxp_status mxp_create_slab(const mxp_grid *grid, int64_t row0, int64_t nrows, const double *c_slab_host,
                           const double *c_range, int device, void *cuda_stream, mxp_problem **out);

/* One Taylor-Horner step of the exp / psi actions (Def. psi, Horner form of the
 * sub-stepped Taylor polynomial), complex128:
 *   out = rho (y + sigma (A_s - mu I) p + gamma v),
 * with the problem's shift mu (mxp_get_plan) and complex scalars sigma, gamma,
 * rho given as {re, im}; y and v nullable (v needs gamma).  One launch on the
 * problem's stream; out must not alias p, y or v. */
mxp_status mxp_horner_step(mxp_problem *prob, const double *sigma, const double *gamma, const double *rho,
                           const void *p_dev, const void *y_dev, const void *v_dev, void *out_dev);

/* The shift mu and the Taylor plan (S sub-steps of degree m) of action `which`
 * (0 exp, 1 psi_1, 2 psi_2) for the current parameters: exp(i t A_s) v =
 * e^{i t mu} (prod over S sub-steps of the degree-m Taylor polynomial of
 * i t (A_s - mu) / S) v. */
mxp_status mxp_get_plan(const mxp_problem *prob, int which, double *mu, int *S, int *m);

/* Vector operations of a Krylov solve split over slabs (one per rank), on
 * complex128 vectors of the problem's size (its unknowns; for a slab, the
 * extended slab).  Both run on the problem's stream.
 *
 * mxp_vec_mdot: out_host[2i], out_host[2i + 1] = Re, Im of the sum over the
 * rows [row_lo, row_hi) of the last axis (local row indices) of conj(V_i) w,
 * for the k <= 64 vectors V_i = V_dev + i ldv (ldv in complex elements, at
 * least the number of unknowns when k > 1).  FP64, deterministic.  A slab sums
 * the rows it owns and the caller adds the ranks' results (one all-reduce).
 * Synchronises the stream.
 *
 * mxp_vec_combine: y = beta y + sum_{i < k} coef_i V_i, complex scalars as
 * {re, im} (beta[2], coef_host[2k]), 0 <= k <= 64; with beta = 0, y is not read
 * (it may hold anything, NaN included); y must not alias a V_i.
 * Asynchronous (the coefficients are copied before the call returns).
 * MXP_EINVAL for out-of-range k, rows or ldv. */
mxp_status mxp_vec_mdot(mxp_problem *prob, const void *V_dev, int64_t ldv, int k, const void *w_dev,
                        int64_t row_lo, int64_t row_hi, double *out_host);
mxp_status mxp_vec_combine(mxp_problem *prob, void *y_dev, const double *beta, const void *V_dev, int64_t ldv,
                           int k, const double *coef_host);

/* Fill *p with the paper's rules for a grid whose slowest speed is c_min and
 * `ppw` points per slowest wavelength: omega = 2 pi c_min / (ppw h),
 * freq = 1/(ppw h), s = 1/freq, t = 40 h^2 (0.4/freq^2 at ppw 10), C_pml 20,
 * fprtol 0.08, exp_tol 1e-12, restart 30 (Sec. 4). */
mxp_status mxp_default_params(const mxp_grid *grid, double c_min, double ppw,
                              mxp_params *p);

/* Replace the problem's parameters (NULL restores the defaults). */
mxp_status mxp_set_params(mxp_problem *prob, const mxp_params *p);
mxp_status mxp_get_params(const mxp_problem *prob, mxp_params *p);

/* Boundary condition of one face of the grid. */
typedef enum {
    MXP_BC_DIRICHLET = 0,   /* zero value beyond the grid (default; used with a PML) */
    MXP_BC_SOUND_HARD = 1,  /* du/dn = 0 through a ghost point: u_ghost = u_p */
    MXP_BC_ABSORBING = 2    /* first-order absorbing du/dn = i k u, k = omega / c_p:
                               u_ghost = u_p (1 + i k h/2) / (1 - i k h/2) */
} mxp_bc;

/* Face conditions of the problem: bc[6] for the faces x-, x+, y-, y+, z-, z+
 * (faces beyond the grid's dimension must be MXP_BC_DIRICHLET).  These are the
 * mixed boundary conditions of the Marmousi-II case of Sec. 4 (a sound-hard
 * surface and first-order absorbing sides and bottom, discretised with ghost
 * points; normally with npml = 0).  The face lies midway between a boundary
 * unknown and its ghost; the ghost's coefficient joins the diagonal of the
 * boundary rows of A and A_s.  With any non-Dirichlet face the exp / psi
 * actions run on kernels that carry these face terms: in 2D (complex64 and
 * bfloat16 storage) the persistent exp-action kernel when one of its face
 * configurations fits the grid, otherwise the per-point sweep; the tiled
 * per-pass kernels (fused 2D, z-marching 3D) assume zero ghosts and are not
 * used.  Copies bc; allocates the face terms on the problem's device
 * (MXP_ENOMEM on failure); MXP_EINVAL for an unknown code. */
mxp_status mxp_set_boundary(mxp_problem *prob, const int *bc);
mxp_status mxp_get_boundary(const mxp_problem *prob, int *bc);

/* y = A x (shifted = 0) or y = A_s x (shifted = 1), complex128.
 * (A x)_p = sum_d a_d [b_d+ (x_{p+e_d} - x_p) - b_d- (x_p - x_{p-e_d})] / h^2
 *           + omega^2 (1 + i s [shifted]) / c_p^2 x_p, with a_d = 1/s_d at the
 * node and b_d+- = 1/s_d at the half nodes (Eq. helmholtz, Eq. pml-1d-s,
 * Sec. 3.4).  Always computed in FP64. */
mxp_status mxp_apply_operator(mxp_problem *prob, int shifted, const void *x_dev,
                              void *y_dev);

/* y = exp(i t A_s) x (which = 0), psi_1(i t A_s) x (which = 1) or
 * psi_2(i t A_s) x (which = 2) (Def. psi), in the problem's precision; x and y
 * are complex128.  psi_1 and psi_2 are read off the exponential of the matrix
 * augmented by one scalar row (psi_1) or a 2x2 Jordan block (psi_2).
 * passes_out (nullable) receives the number of stencil sweeps.  MXP_EINVAL for
 * any other which. */
mxp_status mxp_apply_phi(mxp_problem *prob, int which, const void *x_dev, void *y_dev,
                         int64_t *passes_out);

/* w = MatExPre(r): Algorithm 1 with the problem's parameters (P_N r when
 * params.precond = 1, st->inner_iters then reporting N; the second inverse
 * formula's variant when params.precond = 2).  st nullable.
 * Returns MXP_OK also when the inner GMRES stopped at inner_maxit (st->converged
 * tells which); MXP_ENAN if a residual became non-finite. */
mxp_status mxp_apply_matexpre(mxp_problem *prob, const void *r_dev, void *w_dev,
                              mxp_apply_stats *st);

/* Solve A x = b (unshifted A) by FGMRES(restart) preconditioned on the right
 * by MatExPre (Sec. 3.4).  Returns MXP_ENOCONV when maxit is reached first
 * (x then holds the last iterate).  st nullable.  b = -f for Eq. helmholtz. */
mxp_status mxp_solve(mxp_problem *prob, const void *b_dev, void *x_dev,
                     const mxp_solve_opts *opts, mxp_solve_stats *st);

/* mxp_solve with HOST buffers: copies b to the device, solves, copies x back
 * (x_host also supplies the initial guess when opts->x0_given). */
mxp_status mxp_solve_host(mxp_problem *prob, const void *b_host, void *x_host,
                          const mxp_solve_opts *opts, mxp_solve_stats *st);

/* Many right-hand sides over several problems in one call.  Right-hand side r
 * belongs to problem probs[prob_of_rhs[r]]; b_dev[r], x_dev[r] are its vectors
 * on that problem's device.  Scheduling:
 *  - 2D problems in MXP_C64 or MXP_BF16S without faces (Algorithm 1) with
 *    fewer than 2^20 unknowns form one group on one device: the sources of all
 *    of them advance in lockstep (outer FGMRES and inner GMRES side by side),
 *    every pass of their exp / psi_1 actions is one launch over all active
 *    sources, converged sources are masked on the device, and each action's
 *    pass sequence is replayed from a captured CUDA graph;
 *  - a 2D problem whose actions run on the persistent kernel and that has at
 *    least 2^20 unknowns solves its sources one after another with the
 *    single-source FGMRES (as mxp_solve): there the persistent kernel fills the
 *    GPU and the lockstep batch would be slower;
 *  - any other problem advances its own sources in lockstep, one host thread
 *    per problem, concurrently with the group (kernels overlap when the
 *    problems were created on different streams); problems whose actions run on
 *    the persistent kernel run after that, one at a time.
 * The lockstep paths require precond = 0, and their inner GMRES stops after
 * inner_restart iterations if fprtol is not met.  per_rhs (nullable) has nrhs
 * entries.  Returns MXP_ENOCONV if some source reached maxit. */
mxp_status mxp_solve_batch(mxp_problem *const *probs, int nprob, int nrhs,
                           const int *prob_of_rhs, const void *const *b_dev,
                           void *const *x_dev, const mxp_solve_opts *opts,
                           mxp_solve_stats *per_rhs);

/* Number of fused 2D tile configurations, and the sweep kernel the problem
 * currently uses: -1 = unfused, else a configuration index whose fused step
 * count is returned in *fuse_k (nullable). */
int mxp_num_tile_configs(void);

/* Number of persistent 2D configurations (valid values of persist_cfg). */
int mxp_num_persist_configs(void);
int mxp_tile_config(const mxp_problem *prob, int *fuse_k);
/* Persistent exp-action kernel in use (-1 = none) and its tile count. */
int mxp_persist_config(const mxp_problem *prob, int *ntiles);
/* Its tiles: extents txo x tyo, counts ntx x nty (one CTA each) and the steps
 * K per exchange (each CTA updates its tile plus a K-cell ring); returns the
 * configuration (-1 = none, extents then 0) or -1 for a NULL argument. */
int mxp_persist_geometry(const mxp_problem *prob, int *txo, int *tyo, int *ntx, int *nty, int *k);

/* Kernel that runs the exp-action sweeps of the problem (the choice of the
 * autotuner and of the grid; no counterpart in the paper). */
typedef enum {
    MXP_SWEEP_POINTWISE = 0,      /* one launch per Taylor step, one thread per unknown */
    MXP_SWEEP_FUSED_2D = 1,       /* K steps per launch on shared-memory tiles */
    MXP_SWEEP_PERSISTENT_2D = 2,  /* one cooperative launch per action, grid held on chip */
    MXP_SWEEP_FUSED_3D = 3,       /* K steps per launch by z-marching temporal blocking */
    MXP_SWEEP_ZMARCH_3D = 4,      /* one launch per step, threads march along z in registers */
    MXP_SWEEP_ZMARCH_TMA_3D = 5   /* one launch per step, planes staged by TMA (n0 % 4 == 0) */
} mxp_sweep_kind;
/* Returns an mxp_sweep_kind, or -1 for a NULL problem or a failed set-up.
 * For 3D low-precision problems it may allocate the problem's work buffers and
 * build their TMA descriptors (as the first action would). */
int mxp_sweep_kernel(mxp_problem *prob);

/* Taylor plan of the exp / psi actions (host only, no device call): for a
 * bound nu on ||t (A_s - mu)|| (shifted operator, Sec. 3.4) the number of
 * sub-steps S >= nu / theta_max and the degree m per sub-step, a multiple of
 * kmult, that minimise S m subject to the remainder bound
 * S (nu/S)^(m+1) / (m+1)! e^(nu/S) <= tol.  Returns 1, or 0 for invalid
 * arguments (outputs then unchanged).  No counterpart in the paper, which uses
 * SLEPc's Krylov method for these actions. */
int mxp_taylor_plan(double nu, double tol, double theta_max, int kmult, int *S, int *m);

/* Tile planner of the persistent exp-action kernel (host only, no device
 * call; the paper has no counterpart).  Splits an n0 x n1 grid into at most
 * `slots` tiles of at most txmax x tymax cells, minimising the region (tile
 * plus a k-cell ring) per CTA, with every tile but the last of each row and
 * column at least k cells wide, so that a tile's ring lies inside its eight
 * neighbours.  Writes the tile extents and the tile counts per axis; returns 1,
 * or 0 when no plan fits or an argument is invalid (outputs then unchanged). */
int mxp_persist_tile_plan(int n0, int n1, int slots, int k, int txmax, int tymax,
                          int *txo, int *tyo, int *ntx, int *nty);

/* Allocation-free exp / psi_1 action.  The paper has no counterpart: this is
 * a service for callers that cannot allocate device memory when they need an
 * action -- plugins whose host application owns all device memory through its
 * own pool, or loops that cannot afford a cudaMalloc (which may synchronise the
 * device).
 *
 * Computes y = exp(i t A_s) x (which = 0) or y = psi_1(i t A_s) x (which = 1)
 * in complex128 with the shift and Taylor plan of mxp_apply_phi (prec =
 * MXP_C128; the same host planning code), without a problem handle: grid and
 * params (omega, c_pml, shift_s, t, exp_tol, theta_max; the other fields are
 * ignored) describe the problem, c_dev is the wave speed on the device
 * (prod_d n_d doubles, x fastest, finite and > 0, else MXP_EINVAL), x_dev /
 * y_dev are caller-owned complex128 device vectors (not aliased), work is
 * ordered on cuda_stream (NULL = legacy default stream).  Every call copies the
 * range of c to the host and synchronises the stream once, since the shift and
 * the plan are chosen on the host from it.
 *
 * All workspace lives in one fixed device array compiled into the library:
 * at most 262,144 unknowns, 4,096 unknowns per axis and 64 PML cells per side
 * (about 16 MB, held by every GPU that loads the library until the process
 * exits).  Larger grids return MXP_EINVAL with a message in mxp_last_error().
 * The call makes no device allocation.  Calls share the array: calls whose
 * work overlaps on the GPU (other streams, other host threads) race and must be
 * ordered by the caller.  The first call on a device looks up the array's
 * device address. */
mxp_status mxp_apply_phi_noalloc(const mxp_grid *grid, const mxp_params *params,
                                 const double *c_dev, int which, const void *x_dev,
                                 void *y_dev, void *cuda_stream, int64_t *passes_out);

/* ---------------------------------------------------------------- learned stage
 * A six-layer U-Net-style CNN (bfloat16 weights, float32 accumulation) with
 * GPU training and inference kernels, used as an extra FGMRES preconditioning
 * stage with MatExPre as fallback.  The paper has no learned stage; this is an
 * extension of this library.  Tensors are float32 NCHW device arrays: input
 * channels (Re r, Im r, c / c_max) with r scaled to unit root-mean-square,
 * output channels (Re z, Im z).  H and W must be even.
 * Layers: 3->32 relu; 32->64 stride 2 relu; 64->64 relu; 64->64 relu;
 * nearest x2 upsample then 64->32 relu plus the first layer's output (skip);
 * 32->2.  Flat parameters (float32): W1, b1, ..., W6, b6 with W as
 * [c_out][c_in][3][3]. */
typedef struct mxp_cnn mxp_cnn;
int64_t mxp_cnn_num_params(void);
/* Buffers sized for batches up to max_batch of max_h x max_w images. */
mxp_status mxp_cnn_create(int device, void *cuda_stream, int max_batch, int max_h, int max_w,
                          mxp_cnn **out);
/* Set the float32 master parameters (host array) and reset the Adam state. */
mxp_status mxp_cnn_set_params(mxp_cnn *net, const float *host_params);
mxp_status mxp_cnn_get_params(const mxp_cnn *net, float *host_params);
/* y = network(x) for N images of H x W. */
mxp_status mxp_cnn_forward(mxp_cnn *net, int N, int H, int W, const float *x_dev, float *y_dev);
/* Parameter gradient of sum(gy * y) for the last forward (whose input was x_dev). */
mxp_status mxp_cnn_backward(mxp_cnn *net, const float *x_dev, const float *gy_dev, float *grad_dev);
/* One Adam step (lr, beta 0.9 / 0.999) on the mean squared error between the
 * network output for x and target; *loss_out (nullable) receives the loss. */
mxp_status mxp_cnn_train_step(mxp_cnn *net, int N, int H, int W, const float *x_dev,
                              const float *target_dev, float lr, float *loss_out);
void mxp_cnn_destroy(mxp_cnn *net);
/* One 3x3 convolution of the network's kind on the tensor cores (tcgen05,
 * bfloat16 operands, float32 accumulation), the building block of the
 * learned stage exposed on its own.  Zero padding 1; the logical input is
 * Hl x Wl = Hs x Ws, or 2 Hs x 2 Ws nearest-upsampled when upsample = 1
 * (stride 1 only); Ho = ceil(Hl / stride), Wo = ceil(Wl / stride).  Float32 NCHW
 * device arrays, weights W [Cout][Cin][3][3] as bfloat16 bits.
 *  mode 0 (forward):   out [N][Cout][Ho][Wo] = act(bias + conv(a)), a = the input
 *                      [N][Cin][Hs][Ws] rounded to bfloat16, act = relu when
 *                      relu != 0, bias nullable; Cout <= 64.
 *  mode 1 (input gradient, upsample = 0): out [N][Cin][Hs][Ws] = the gradient
 *                      of sum(g * conv(x)) w.r.t. x, a = g [N][Cout][Ho][Wo]
 *                      rounded to bfloat16; Cin <= 64.
 *  mode 2 (weight gradient): out [Cout][Cin * 9] = the gradient w.r.t. W, a = x
 *                      [N][Cin][Hs][Ws], b = g [N][Cout][Ho][Wo], both rounded to
 *                      bfloat16; Cout <= 64; out is overwritten.
 * Work is ordered on cuda_stream, which the call synchronises once (to read the
 * kernels' wait status: MXP_ETIMEOUT if a bounded wait gave up).  MXP_EINVAL
 * for inconsistent sizes.  No counterpart in the paper. */
mxp_status mxp_cnn_conv3x3(int mode, int stride, int upsample, int N, int Cin, int Hs, int Ws, int Cout,
                           int Ho, int Wo, const float *a_dev, const float *b_dev, const void *w_bf16_dev,
                           const float *bias_dev, int relu, float *out_dev, void *cuda_stream);

/* Use net as the first preconditioner of every FGMRES iteration of prob (2D):
 * the direction z = net(v) is kept when the scaled residual
 * min_a ||v - a A z|| / ||v|| <= accept_tol, otherwise MatExPre(v) is used.
 * net = NULL detaches.  The network must accept the grid's n_y x n_x images. */
mxp_status mxp_attach_cnn(mxp_problem *prob, mxp_cnn *net, double accept_tol);

/* Failure-detection self-test (no counterpart in the paper): launches the
 * bounded device-side wait used by the persistent kernel's grid barrier with an
 * arrival that never happens; the wait gives up after a few thousand polls and
 * sets the problem's error word.  When the problem uses the persistent
 * exp-action kernel, one such action (on the problem's work buffers) follows
 * before the host reads the word, which shows that a later launch keeps the
 * error of an earlier one.  The call returns MXP_ETIMEOUT and the problem stays
 * usable afterwards. */
mxp_status mxp_selftest_barrier_timeout(mxp_problem *prob);

/* Measured FMA throughput of `device` in flop/s (2 flops per fused
 * multiply-add): *fp32_flops for float, *fp64_flops for double.  Independent
 * FMA chains on every SM, timed with CUDA events (best of three after a
 * warm-up launch); no clock or power setting is touched.  These are the
 * arithmetic ceilings of the rooflines of the sweep kernels that run from
 * on-chip memory and of the complex128 path.  Allocates and frees a small
 * device buffer; synchronises the device.  No counterpart in the paper. */
mxp_status mxp_measure_fma_peak(int device, double *fp32_flops, double *fp64_flops);

/* Number of unknowns prod_d n_d of the problem. */
int64_t mxp_num_unknowns(const mxp_problem *prob);

/* Number of CUDA kernels this library has launched in this process so far
 * (all problems, all devices); for accounting in benchmarks. */
int64_t mxp_kernel_launch_count(void);

void mxp_destroy(mxp_problem *prob);
const char *mxp_status_string(mxp_status s);
const char *mxp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MATEXPRE_H */
