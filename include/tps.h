/*
 * tps.h -- C ABI of the GB300 tensor-product three-body eigensolver.
 *
 * Implements the hot path of "Tensor Product Scheme for Computing Bound States
 * of the Quantum Mechanical Three-Body Problem" (arXiv 2111.02534):
 * the pseudospectral Jacobi-coordinate Hamiltonian applied to blocks of wave
 * functions as dense mode products plus a pointwise potential (Sec. 3.2-3.3),
 * the shifted kinetic preconditioner (Sec. 4.2) and the block Jacobi-Davidson
 * eigensolver around them (Sec. 4.1).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Units: hbar and the masses are given explicitly (tps_set_masses), or the
 *    paper's heavy-light units are selected with tps_set_alpha.  The kinetic
 *    coefficient of coordinate k is a_k = -hbar^2 / (2 mu_k); x is the
 *    heavy-heavy separation (mu_x = M/2), y the light particle relative to the
 *    heavy pair's centre of mass (mu_y = 2Mm/(2M+m)).
 *  - Grid: each coordinate is a periodic Fourier grid x_j = -L + j*2L/n on
 *    [-L, L), n even and >= 4; D2 is the dense spectral second derivative.
 *  - Vectors: FP64, one wave function after another.  1D layout [nvec][n_x][n_y],
 *    2D layout [nvec][n_x1][n_x2][n_y1][n_y2], the last index fastest (the
 *    ordering of Sec. 3.1).  N = product of the n's.
 *  - Pointers named *_dev are device pointers on the context's device; *_host are
 *    host pointers.  The caller owns every buffer it passes; the context owns
 *    every device array it allocates (operators, potential, workspaces) and
 *    frees them in tps_destroy.  Apply calls never allocate.
 *  - Calls taking a stream are asynchronous on it unless stated otherwise;
 *    stream 0 is the legacy default stream.
 *  - Every call returns a tps_status; on failure tps_last_error(ctx) describes it.
 *    No exception crosses the ABI.  A context is not thread-safe.
 */
#ifndef TPS_H
#define TPS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *cudaStream_t; /* identical to the CUDA runtime's typedef */

typedef struct tps_ctx tps_ctx;

typedef enum tps_status {
  TPS_OK = 0,
  TPS_ERR_INVALID_ARG = -1,   /* a size, pointer, enum or value is out of range */
  TPS_ERR_NOT_CONFIGURED = -2,/* masses, grid or potential not set yet */
  TPS_ERR_CUDA = -3,          /* a CUDA runtime call failed (message has the CUDA error) */
  TPS_ERR_NOMEM = -4,         /* a device allocation failed */
  TPS_ERR_SINGULAR = -5,      /* the preconditioner's shift hits the kinetic spectrum */
  TPS_ERR_NOT_CONVERGED = -6, /* solver hit its iteration cap; results valid for stats->n_converged pairs */
  TPS_ERR_TIMEOUT = -7        /* a bounded device wait expired (tps_device_status, tps_solve) */
} tps_status;

enum { TPS_GAUSS = 0, TPS_LORENTZ3 = 1 };          /* f_G = exp(-xi^2), f_L = (1+xi^2)^-3 */
enum { TPS_ANY = 0, TPS_X_EVEN = 1, TPS_X_ODD = 2 }; /* heavy-exchange sector (Sec. 5.1) */
enum { TPS_F64 = 0, TPS_F32 = 1, TPS_F64_TC = 2, TPS_TF32_TC = 3 };  /* arithmetic of apply calls
                                                                       (data stay FP64) */
/* TPS_F64_TC: FP64-accurate mode products emulated on the BF16 tensor cores by error-free
 * splitting into digit slices per operand row (1D: 9 six-bit digits for the wave function,
 * 10 for the mode matrices; 2D, at most 128 points per mode: 7 and 8 eight-bit digits;
 * Ozaki scheme), exact FP32 accumulation per digit level, FP64 recombination; H-apply only.
 * TPS_TF32_TC: the preconditioner's mode products on the tensor cores with TF32 inputs
 * (10 explicit mantissa bits) and FP32 accumulation, ~2.5e-3 relative to the exact
 * (T - sigma)^-1 r; preconditioner only (1D; 2D when every mode has 4 to 128 points, a
 * multiple of 4). */
/* Rayleigh-Ritz eigensolver (Sec. 4.1, the projected problem G y = theta y, m <= 64):
 * TPS_RR_MIXED: FP32 eigenvectors (tridiagonalisation, bisection, inverse iteration), then FP64
 *   iterative refinement of the eigenvectors
 *   (Ogita-Aishima, with close eigenvalues rotated as groups) to the same accuracy as
 *   TPS_RR_JACOBI64, which the same launch runs instead if the refinement stalls;
 * TPS_RR_JACOBI64: cyclic Jacobi in FP64. */
enum { TPS_RR_MIXED = 0, TPS_RR_JACOBI64 = 1 };

/* ---- context ------------------------------------------------------------ */

/* Create a context for a 1D (dim = 1) or 2D (dim = 2) three-body problem on CUDA
 * device `device`.  Sec. 2: the three-body problem in d dimensions is a
 * 2d-dimensional eigenvalue problem after removing the centre of mass. */
int tps_create(tps_ctx **out, int dim, int device);
int tps_destroy(tps_ctx *ctx);
const char *tps_last_error(const tps_ctx *ctx);
const char *tps_status_string(int status);
/* Synchronise the context's device and report whether a tensor-core kernel of this
 * context gave up a bounded wait since the last call (TPS_ERR_TIMEOUT; its outputs are
 * then invalid) -- each such wait ends after about one second instead of hanging. */
int tps_device_status(tps_ctx *ctx);
/* Self-test of that failure path: a one-warp kernel waits on a barrier that nothing
 * signals, gives up after `seconds` (0 < seconds <= 2) exactly as the tensor-core kernels'
 * waits do, and records it; a second kernel then checks that the device still takes work.
 * Returns TPS_ERR_TIMEOUT when both happened (the expected outcome), TPS_ERR_CUDA
 * otherwise.  Synchronous; allocates and frees 8 bytes. */
int tps_selftest_wait_timeout(int device, double seconds);

/* ---- problem definition ------------------------------------------------- */

/* Sec. 2 (Eq. Schroedinger_equation_three_body): kinetic coefficients from the
 * heavy mass M, light mass m and hbar (all > 0).  a_x = -hbar^2/M,
 * a_y = -hbar^2 (2M+m) / (4Mm). */
int tps_set_masses(tps_ctx *ctx, double M, double m, double hbar);

/* Sec. 2: the paper's dimensionless form, heavy-light reduced mass 1:
 * a_x = -alpha_x/2 = -1/(1+alpha), a_y = -alpha_y/2 = -(1+2alpha)/(4+4alpha). */
int tps_set_alpha(tps_ctx *ctx, double alpha);

/* Sec. 3.1: grid sizes n[0..2*dim-1] (each even, >= 4) and half box lengths
 * L[0..2*dim-1] (> 0), order (x, y) or (x1, x2, y1, y2), host arrays.  Builds the
 * dense operators a_k*D2_k and their eigendecompositions on the device.  In 2D
 * n_x1 = n_x2 and n_y1 = n_y2 (with equal L) are required. */
int tps_set_grid(tps_ctx *ctx, const int *n, const double *L);

/* Sec. 3.1, the paper's own discretisation (1D contexts): each coordinate on the n[k]
 * roots of the Chebyshev polynomial T_n mapped to the real line by y = L t / sqrt(1 - t^2)
 * (tps_chebyshev_grid), with the dense non-symmetric D2 there; n[k] even in [4, 1024],
 * L[k] > 0 (the map parameter).  Replaces the Fourier grid of tps_set_grid.  Builds the
 * operators a_k D2_k, their eigen-decompositions D2 = S diag(lam) S^-1 (a real spectrum;
 * TPS_ERR_SINGULAR otherwise) for the Sec. 4.2 preconditioner, which then applies S^-1 where
 * the Fourier grid applies S^T.  Pair potentials are evaluated at the mapped points; the
 * heavy-exchange sectors fold the mirror-image nodes x_i = -x_{n-1-i}; tps_solve runs a
 * Jacobi-Davidson method for non-symmetric H (Ritz pairs of the non-symmetric projected
 * matrix, Sec. 4.1); tps_apply_prec accepts TPS_F64 and TPS_F32 only. */
int tps_set_grid_chebyshev(tps_ctx *ctx, const int *n, const double *L);

/* Sec. 3.3 (Eq. tensor_form): an arbitrary diagonal potential V[N] in the vector
 * layout (no structure assumed), copied in.  on_device != 0: V is a device
 * pointer, else a host pointer.  Requires tps_set_grid first. */
int tps_set_potential(tps_ctx *ctx, const double *V, int on_device);

/* Eq. definition_potential: V = -v0 [f(|y - x/2|/sigma) + f(|y + x/2|/sigma)]
 * (2D: vector distances), evaluated pointwise on the grid.  shape TPS_GAUSS or
 * TPS_LORENTZ3, sigma > 0. */
int tps_set_pair_potential(tps_ctx *ctx, int shape, double v0, double sigma);

/* Sec. 2 and Sec. 5.1: the smallest well depth v0 for which the two-body problem
 * [-hbar^2/(2 mu_hl) Laplacian - v0 f(|xi|/sigma)] psi = -E0 psi has a solution,
 * from the generalized eigenvalue problem (T + E0) psi = v0 F psi on the periodic
 * grid with n points per dimension on [-L, L) (dim 1 or 2).  E0 > 0.  Host-side
 * setup computation; writes *v0_out. */
int tps_two_body_v0(int dim, double mu_hl, double hbar, double E0, int shape, double sigma,
                    int n, double L, double *v0_out);

/* Sec. 3.1, the paper's own discretisation of one coordinate: collocation on the n roots
 * of the Chebyshev polynomial T_n, t_j = -cos(pi (j + 1/2) / n) (ascending), mapped to the
 * real line by the algebraic map y = L t / sqrt(1 - t^2), and the second-derivative
 * matrix there, D2 = diag((dt/dy)^2) D D + diag(d^2t/dy^2) D with D the derivative of the
 * polynomial interpolant on the roots (dense and non-symmetric).  Host-side setup
 * computation: writes y_host[n] and D2_host[n * n] (row-major); 2 <= n <= 1024, L > 0,
 * else TPS_ERR_INVALID_ARG.  With lam_host, S_host and Sinv_host non-null it also writes
 * the fast-diagonalisation factors of the Sec. 4.2 preconditioner on this grid,
 * D2 = S diag(lam) S^-1 (lam ascending, unit columns of S, row-major), from a host QR
 * eigensolver; TPS_ERR_SINGULAR if D2 has a complex pair or S is singular.  A context
 * takes this grid through tps_set_grid_chebyshev. */
int tps_chebyshev_grid(int n, double L, double *y_host, double *D2_host, double *lam_host,
                       double *S_host, double *Sinv_host);

/* Tile autotuning of the mode-product GEMMs (on by default, process-wide): the first
 * launch of each GEMM shape times the candidate tile shapes on the caller's stream (which
 * adds a host synchronisation to that first call) and later launches use the fastest.
 * Results are bitwise identical for every tile shape.  Skipped during stream capture. */
int tps_set_autotune(int on);

/* Number of unknowns N and the norm estimate ||H||_est = sum_k |a_k| (pi/h_k)^2 + max|V|. */
int tps_get_info(const tps_ctx *ctx, long long *N, double *hnorm_est);

/* ---- hot path: operator applications ----------------------------------- */

/* Eq. tensor_op1D (1D) and Eq. tensor_op2D (2D): out = (H - theta) psi for nvec
 * vectors, H = sum_k a_k (I x .. x D2_k x .. x I) + diag(V).  psi_dev, out_dev:
 * device, [nvec][N] FP64, must not overlap.  dtype TPS_F64: FP64 arithmetic; TPS_F32:
 * FP32 arithmetic (error ~ n eps_32 ||H|| |psi|), the low-precision phase's operator;
 * TPS_F64_TC: FP64-accurate products on the tensor cores (error below
 * 2^-53 n of row max x column max per product, like FP64 arithmetic).  The first
 * TPS_F64_TC call on a context builds the operator's digit slices (a few MB) and a
 * slice workspace of up to 256 MB (2D: the four mode products one after the other, a
 * fiber-slice workspace of up to 1 GB; TPS_ERR_INVALID_ARG for more than 128 points in a
 * mode). */
int tps_apply_h(tps_ctx *ctx, const void *psi_dev, void *out_dev, int nvec, double theta,
                int dtype, cudaStream_t stream);

/* Sec. 4.2 (Eq. sylvester_equation): out = (T - theta)^-1 r, T the kinetic part of
 * H (V neglected), by fast diagonalisation S ((S^T r S) ./ (Lambda (+) .. - theta)) S^T
 * over all 2*dim modes.  Returns TPS_ERR_SINGULAR when
 * min |lambda_sum - theta| < 1e-14 * max |lambda_sum|.  r_dev, out_dev: device
 * [nvec][N] FP64, must not overlap.  dtype TPS_F64: FP64 arithmetic; TPS_F32: FP32
 * arithmetic; TPS_TF32_TC: the mode products (four in 1D, eight in 2D) on the tensor
 * cores with TF32 inputs and FP32 accumulation, ~2.5e-3 relative to the exact solve (the
 * first call on a context builds padded FP32 eigenbases of a few MB); in 2D every mode
 * must have 4 to 128 points, a multiple of 4 (else TPS_ERR_INVALID_ARG).  The
 * preconditioner only approximates (H - theta)^-1 whatever the dtype: the solver uses
 * TPS_TF32_TC by default (TPS_F32 on 2D grids it does not take). */
int tps_apply_prec(tps_ctx *ctx, const void *r_dev, void *out_dev, int nvec, double theta,
                   int dtype, cudaStream_t stream);

/* ---- hot path: solver ---------------------------------------------------- */

typedef struct tps_solver_opts {
  int m_min;          /* search-space size kept at restart (0: max(2k, 8) rounded up to the block) */
  int m_max;          /* search-space size that triggers a restart (0: m_min + 2*block; at most 64) */
  int inner_steps;    /* GMRES steps per correction equation (Sec. 4.1).  0: adaptive -- one
                         step (the correction is the projected preconditioned residual
                         -Kt^-1 r), widened to 3, 7, 10 when the outer residual stalls */
  int max_outer;      /* outer-iteration cap (0: 500) */
  int use_prec;       /* 1: prec-JDQR (Sec. 4.2 preconditioner), 0: no-prec-JDQR */
  double prec_shift;  /* fixed preconditioner shift (the paper's -E0); NaN: adaptive, -|theta| of
                         the lowest active Ritz value (kept below the kinetic spectrum) */
  unsigned long long seed; /* start block when x0 is NULL (counter-based normal deviates) */
  double inner_tol;   /* GMRES stops a system when its preconditioned residual drops by this
                         factor (0: 1e-3) */
  int timing;         /* 1: time every H and preconditioner application with CUDA events on
                         the solve's stream (tps_stats h_ms / prec_ms) */
  int guard;          /* extra eigenpairs converged beyond k and discarded, so that a state
                         absent from the early search space is not skipped (default 2) */
  int smooth_start;   /* applications of the kinetic preconditioner (shift -1e-3 ||H||_est) to
                         the random part of the start block, a low-pass filter (default 2) */
  int prec_dtype;     /* arithmetic of the preconditioner inside the solver: TPS_TF32_TC
                         (default; tensor cores -- TPS_F32 on 2D grids whose modes are not
                         4 to 128 points, a multiple of 4), TPS_F32 or TPS_F64 */
  int h_dtype;        /* TPS_F64 (default): FP64 H products throughout (on the tensor cores,
                         see h64_dtype); TPS_F32: mixed precision -- a first phase runs the H
                         mode products in FP32 until every pair's residual is below
                         switch_tol, then an FP64 refinement phase converges them to tol.
                         Gram matrices, Ritz values and QR steps are FP64 always */
  double switch_tol;  /* relative residual ending the FP32 phase (0: 1e-6) */
  int refine_block;   /* block size of the FP64 refinement phase (0: k + guard, at most 32) */
  int refine_inner_steps; /* GMRES steps in the refinement phase (0: adaptive as above) */
  int refine_inner_dtype; /* arithmetic of H inside the refinement's GMRES (TPS_F64 default) */
  int h64_dtype;      /* how every FP64 H-apply of the solver runs (refinement phase, FP64-only
                         mode, final Rayleigh quotients): TPS_F64_TC (default: tensor-core
                         emulation; 2D grids with more than 128 points in a mode use the FMA
                         pipe) or TPS_F64 (FMA pipe) */
  int rr_method;      /* Rayleigh-Ritz eigensolver: TPS_RR_MIXED (default) or TPS_RR_JACOBI64 */
  int rr_refine_max;  /* TPS_RR_MIXED: FP64 refinement iterations before the FP64 Jacobi
                         takes over (0: 12) */
  int correction_dtype; /* arithmetic of the Gram and update products inside the correction
                         solve (projectors, GMRES Arnoldi), which is solved to inner_tol and
                         whose result is orthonormalised in FP64 before it enters the basis:
                         TPS_F32 (default) or TPS_F64 */
  int update_dtype;   /* arithmetic of the FP64 block updates of the outer iteration (Ritz
                         vectors, restarts, orthogonalisation; the Cholesky-QR product stays
                         on the FMA pipe): TPS_F64_TC (default: digit-split products on the
                         tensor cores, tps_block_update_tc, for blocks of 10^5 rows or more
                         and p >= 8; smaller ones on the FMA pipe) or TPS_F64 (FMA pipe) */
  int graph;          /* 1: after the host-driven outer iterations that fill the first m_min
                         columns, the rest of the solve runs
                         as one CUDA graph launch: the outer iteration is captured once, with
                         every wanted pair in one block (k <= 16, `block` and `guard` ignored;
                         the search space cycles between m_min (default 4k), rounded up to
                         whole blocks, and m_min + 2k <= 64),
                         no locking, the preconditioner shift prec_shift if given, else set
                         on the device every iteration from the lowest unconverged Ritz value
                         (converged pairs get no correction), and one
                         preconditioned-residual step per correction, inside a conditional
                         WHILE node whose condition a device kernel sets from the residual
                         norms.  Falls back to the host-driven loop if the cycle does not
                         converge within max_outer iterations.  1D Fourier grids, no warm
                         start; ignored otherwise.  Default 0 */
  int gram_dtype;     /* arithmetic of the FP64 Gram products of the outer iteration
                         (orthogonalisation coefficients, Cholesky-QR Grams, the
                         Rayleigh-Ritz matrix): TPS_F64_TC (default: digit-split products on
                         the tensor cores, tps_gram_tc, for blocks of 10^5 rows or more with
                         min(p, q) <= 8 and max(p, q) <= 64; others on the FMA pipe) or
                         TPS_F64 (FMA pipe).  Symmetric solver only */
} tps_solver_opts;

typedef struct tps_stats {
  int outer_iters;    /* Newton (outer) iterations */
  int h_applies;      /* single-vector H applications (MVMs, Table 2) */
  int prec_applies;   /* single-vector preconditioner applications */
  int inner_steps;    /* GMRES steps summed over systems */
  int restarts;
  int n_converged;    /* pairs returned */
  double hnorm_est;
  double time_ms;     /* wall time of tps_solve */
  double h_ms;        /* with opts.timing: device time of the H applications */
  double prec_ms;     /* with opts.timing: device time of the preconditioner applications */
  double h_flops;     /* algorithmic FP64 flops of the H applications (2N(sum n_k) + 3N each) */
  double prec_flops;  /* algorithmic flops of the preconditioner applications (4N(sum n_k) + N) */
  long long h_launches;      /* H-application launches (each over a block of vectors) */
  long long prec_launches;   /* preconditioner-application launches */
  long long kernel_launches; /* all CUDA kernels launched by this call */
  double h32_ms;      /* with opts.timing: device time of the FP32 H applications */
  double h32_flops;   /* algorithmic flops of the FP32 H applications */
  long long h32_launches;
  /* FP64 Gram products A^T B and block updates C = bC + a A Y (a6, a7), with opts.timing
   * (the correction solve's FP32-arithmetic products are not included).  To
   * keep the timing overhead low every 4th launch is timed: *_ms, *_flops and *_bytes
   * cover the timed launches (so flops / ms is their rate), *_launches counts all. */
  double gram_ms;     /* device time of the timed Gram launches */
  double gram_flops;  /* their algorithmic flops, 2 nrows p q each */
  double gram_bytes;  /* their algorithmic bytes, 8 nrows (p + q) each */
  long long gram_launches;
  double upd_ms;      /* device time of the timed block updates */
  double upd_flops;   /* 2 nrows p q each */
  double upd_bytes;   /* 8 nrows (p + q) each, + 8 nrows q when C is read */
  long long upd_launches;
  int jacobi_calls;   /* Rayleigh-Ritz solves by the FP64 cyclic Jacobi (TPS_RR_JACOBI64, or
                         a TPS_RR_MIXED fallback) */
  int jacobi_sweeps;  /* their cyclic Jacobi sweeps, summed */
  int jacobi_rounds;  /* rounds that applied at least one rotation, summed */
  int gs_orthogonalisations; /* block Gram-Schmidt orthogonalisations of new search blocks */
  int gs_second_passes;      /* of which needed a second pass (a column kept < 1/sqrt 2 of
                                its norm after the first) */
  int rr_mixed_calls;        /* Rayleigh-Ritz solves by TPS_RR_MIXED */
  int rr_fp32_solves;        /* their FP32 eigensolves (starting vectors and group rotations) */
  int rr_refine_iters;       /* their FP64 refinement iterations */
  int rr_groups_rotated;     /* groups of close eigenvalues rotated inside the refinement */
  int rr_fallbacks;          /* solves the FP64 Jacobi finished (refinement not converged) */
  double rr_ms;              /* with opts.timing: device time of the Rayleigh-Ritz eigensolves
                                (every 4th launch timed, like the Gram products) */
  long long rr_launches;     /* Rayleigh-Ritz eigensolver launches (all of them) */
  long long rr_timed;        /* of which timed (rr_ms covers these) */
  double graph_build_ms;     /* graph solver: host time to capture and instantiate the graph */
  double graph_run_ms;       /* graph solver: host wall time of the graph launch until done */
  double resid[64];   /* ||H x_i - lambda_i x_i|| / ||H||_est per returned pair */
} tps_stats;

/* Defaults for tps_solve's options. */
void tps_default_opts(tps_solver_opts *opts);

/* Sec. 4.1: the k lowest eigenpairs of H in a heavy-exchange sector (TPS_ANY,
 * TPS_X_EVEN, TPS_X_ODD; 2D supports TPS_ANY only) by block Jacobi-Davidson with
 * block size `block` (1..32; 1 is the paper's single-vector JDQR), converged when
 * ||H x - theta x|| <= tol * ||H||_est.  x0_dev: nullable device [n_x0][N] warm
 * start (Sec. 5.2 homotopy): its first min(n_x0, max(block, k + guard)) columns form the
 * first search block (completed with smoothed random columns up to `block`).
 * evals_host: host [k] ascending.  evecs_dev: device
 * [k][N] unit-norm, sign such that the entry of largest magnitude is positive.
 * opts may be NULL (defaults).  Synchronous: returns when results are ready.
 * The first call allocates the solver's device workspace inside the context
 * (kept for later calls of the same or smaller size).  k <= 64. */
int tps_solve(tps_ctx *ctx, int k, int parity, double tol, int block, const double *x0_dev,
              int n_x0, const tps_solver_opts *opts, double *evals_host, double *evecs_dev,
              tps_stats *stats, cudaStream_t stream);

/* Batched parameter sweep (Sec. 5.2 solves a sequence of problems; the batched sweep
 * over mass ratio and coupling): solves ninst independent problems, instance i described
 * by its own context ctxs[i] (all on one device) with k[i] pairs, concurrently.  nstreams
 * host threads (1..64) each drive a non-blocking CUDA stream of their own and take
 * instances from a shared queue.  evals_host: [ninst][kstride] (k[i] <= kstride);
 * evecs_dev[i]: device [k[i]][N_i]; stats: nullable [ninst]; status: [ninst] per-instance
 * tps_status.  Returns TPS_OK when every instance succeeded, else the first failing status
 * (or TPS_ERR_CUDA if a stream could not be created).  Synchronous.  kernel_launches in
 * the per-instance stats count launches of all instances running at the same time. */
int tps_solve_batch(tps_ctx **ctxs, int ninst, const int *k, int parity, double tol, int block,
                    const tps_solver_opts *opts, double *evals_host, int kstride,
                    double **evecs_dev, tps_stats *stats, int *status, int nstreams);

/* ---- hot path: Jacobi-Davidson building blocks (device FP64) -------------
 * Column blocks are column-major: column c of an nrows x p block A starts at
 * A + c*lda (lda >= nrows).  Small matrices are column-major with leading
 * dimension as given. */

/* Gram matrix G = A^T B (p, q <= 64) -- block orthogonalisation and Rayleigh-Ritz
 * projections of Sec. 4.1.  G_dev: device p x q, leading dimension ldg. */
int tps_gram(tps_ctx *ctx, const double *A_dev, long long lda, int p, const double *B_dev,
             long long ldb, int q, long long nrows, double *G_dev, int ldg, cudaStream_t stream);

/* The same Gram matrix, FP64-accurate, as digit-split BF16 products on the tensor cores
 * (the Ozaki scheme; the solver's default for its FP64 Grams): per block of 64 rows each
 * column of A and of B is scaled by a power of two and its 55-bit integer cut into seven
 * base-256 digits; the digit pairs of levels 0..7 are multiplied exactly, each block's sum
 * is rounded once to FP64 and the blocks are added in FP64.  Error per entry within a small
 * multiple of an FP64 dot product's, 2^-53 (max_r |A[r][i]| sum_r |B[r][j]| + max_r |B[r][j]|
 * sum_r |A[r][i]|) per block of rows.  min(p, q) <= 8 and max(p, q) <= 64, else
 * TPS_ERR_INVALID_ARG; otherwise the same arguments and errors as tps_gram.  The result
 * does not depend on launch scheduling (partial sums added in a fixed order). */
int tps_gram_tc(tps_ctx *ctx, const double *A_dev, long long lda, int p, const double *B_dev,
                long long ldb, int q, long long nrows, double *G_dev, int ldg, cudaStream_t stream);

/* Block update C = beta*C + A Y (p, q <= 64); Y_dev: device p x q, leading
 * dimension ldy.  C must not overlap A. */
int tps_block_update(tps_ctx *ctx, const double *A_dev, long long lda, int p, const double *Y_dev,
                     int ldy, int q, double beta, double *C_dev, long long ldc, long long nrows,
                     cudaStream_t stream);

/* The same block update, FP64-accurate, computed as digit-split BF16 products on the
 * tensor cores (the Ozaki scheme; the solver's default for its FP64 updates): each row of A
 * and each column of Y is scaled by a power of two and its 55-bit integer cut into seven
 * base-256 digits, the digit pairs of levels 0..7 are multiplied exactly and combined in
 * integer arithmetic.  Error per entry at most about 2^-53 max_k |A[r][k]| sum_k |Y[k][j]|.
 * Same arguments, limits and errors as tps_block_update. */
int tps_block_update_tc(tps_ctx *ctx, const double *A_dev, long long lda, int p,
                        const double *Y_dev, int ldy, int q, double beta, double *C_dev,
                        long long ldc, long long nrows, cudaStream_t stream);

/* Orthonormalise the block T (b <= 32 columns) against the orthonormal block Q
 * (nq columns, may be 0) and within itself: two passes of block classical
 * Gram-Schmidt followed by Cholesky QR twice (Sec. 4.1, search-space expansion).
 * Columns that are numerically in span(Q, earlier columns) are set to zero and
 * counted out: *rank_host receives the number of columns kept (the kept columns
 * are moved to the front).  Synchronous. */
int tps_orthonormalize(tps_ctx *ctx, const double *Q_dev, long long ldq, int nq, double *T_dev,
                       long long ldt, int b, long long nrows, int *rank_host, cudaStream_t stream);

/* Eigen-decomposition of a symmetric m x m matrix (m <= 64) on the device (Rayleigh-Ritz
 * of Sec. 4.1) by TPS_RR_MIXED.  theta_dev: m eigenvalues ascending; Y_dev: eigenvectors,
 * column-major m x m with leading dimension ldy.  Off-diagonals of Y^T G Y are left below
 * 8.9e-16 ||G||_F and Y^T Y - I below 4 m 2^-53. */
int tps_small_eigh(tps_ctx *ctx, const double *G_dev, int m, int ldg, double *theta_dev,
                   double *Y_dev, int ldy, cudaStream_t stream);

/* Eq. jdcor with the Sec. 4.2 preconditioner: approximate solutions t_i _|_ Qt of
 * (I - Qt Qt^T)(H - theta_i)(I - Qt Qt^T) t_i = -r_i for nsys systems, by
 * `steps` steps of left-preconditioned GMRES with the projected preconditioner
 * Kt^-1 = K^-1 - K^-1 Qt (Qt^T K^-1 Qt)^-1 Qt^T K^-1, K = T - shift (use_prec = 1),
 * or with the projector alone (use_prec = 0).  Full-grid vectors of this context:
 * Qt_dev [nq][N] orthonormal, R_dev and T_dev [nsys][N], theta_dev [nsys] on the
 * device.  Runs all `steps` steps (a system stops early only on breakdown).
 * nsys <= 32, nq <= 96.  The first call allocates the correction workspace inside
 * the context.  Synchronous. */
int tps_correction(tps_ctx *ctx, const double *Qt_dev, int nq, const double *R_dev,
                   const double *theta_dev, int nsys, int steps, int use_prec, double shift,
                   double *T_dev, cudaStream_t stream);

/* Allocation-free Gram product G = A^T B (p, q <= 64), same layout and result as
 * tps_gram, for callers that cannot allocate device memory: programs whose device
 * memory is owned by a memory manager that hands out all of it up front (a
 * framework's caching allocator, a service with a fixed memory budget).  It needs no
 * context and calls no allocator; its partial sums live in a 1 MiB array compiled into
 * the library, one per device.  The paper has no counterpart to this entry point.
 *  - The first call on each device looks the array's address up (with that device
 *    current) and caches it with the id of the current CUDA context; a call under a new
 *    context (after cudaDeviceReset, for example) looks it up again.  Make the first call
 *    on a device, and the first after a reset, before any stream capture.
 *  - Every call on a device shares the array and it keeps the last call's contents;
 *    calls that overlap on the GPU (e.g. on two streams at once) race on it.
 *  - Returns TPS_ERR_INVALID_ARG for p or q outside 1..64 or bad strides/pointers,
 *    TPS_ERR_CUDA if the address look-up or the launch fails.  Asynchronous on stream. */
int tps_gram_noalloc(const double *A_dev, long long lda, int p, const double *B_dev, long long ldb,
                     int q, long long nrows, double *G_dev, int ldg, cudaStream_t stream);

/* ---- learned warm start (a small MLP trained on the solver's own eigenvectors) ----
 *
 * Along a sweep of binding energies the paper starts each Jacobi-Davidson run from the
 * previous run's subspace (homotopy, Sec. 5.2) and names low-rank vectors as a way
 * forward (Sec. 6).  This model predicts a low-rank separable start block directly from
 * the problem parameters, for any grid.  Inputs: four
 * features of (mass ratio M/m, well depth v0, range sigma, state index) -- see
 * tps_ws_features.  Network: 4 -> [Linear, GELU(exact erf form)] x 3 (width `hidden`) ->
 * Linear -> rank (px + py) outputs read as C (rank x px) and D (rank x py), the state
 *     psi(x, y) = sum_r (sum_a C[r][a] phi_a(x)) (sum_b D[r][b] chi_b(y)),
 * phi_a = cos(a pi x / L_x) (a < px, even under x -> -x), chi_b the real Fourier modes of y
 * (1, cos, sin, cos 2, ...; b < py), both sampled on a context's grid and normalised there.
 * Trained on the GPU (FP32 forward, backward and Adam kernels); inference (tps_ws_predict)
 * runs with BF16 weights.  Parameters: one FP32 array, per layer l = 0..3 the weights
 * W_l[in][out] row-major then the biases b_l[out], layer widths 4, hidden, hidden, hidden,
 * rank (px + py).  Loss per sample against a target T (px x py, from tps_ws_project):
 *     L = 1 - <P, T>^2 / (|P|^2 |T|^2),  P = C^T D,
 * invariant under the arbitrary sign and scale of an eigenvector; the mean over the batch
 * is minimised.  In 2D the same matrix form holds with x and y the Jacobi vectors: psi
 * (layout [x1][x2][y1][y2]) is read as an (n_x1 n_x2) x (n_y1 n_y2) matrix and
 *     phi_a(x) = F_a1(x1) F_a2(x2),  a = a1 q_x + a2,  px = q_x^2,
 * F the real Fourier modes of one Cartesian component (a1, a2 < q_x), chi_b likewise with
 * py = q_y^2; a 2D model needs px and py perfect squares. */
typedef struct tps_ws tps_ws;

/* Create a model on `device` with He-initialised weights (counter-based generator from
 * seed).  px, py <= 128, rank <= 64, hidden <= 4096. */
int tps_ws_create(tps_ws **out, int device, int px, int py, int rank, int hidden,
                  unsigned long long seed);
int tps_ws_destroy(tps_ws *ws);
const char *tps_ws_last_error(const tps_ws *ws);
/* Number of parameters and output width rank (px + py). */
int tps_ws_info(const tps_ws *ws, long long *nparam, int *out_dim);
/* Copy the FP32 parameters out / in (host arrays of exactly nparam floats; synchronous). */
int tps_ws_get_params(tps_ws *ws, float *params_host, long long nparam);
int tps_ws_set_params(tps_ws *ws, const float *params_host, long long nparam);
/* Host feature map, X[i] = (ln(M/m) / ln 40, ln(v0) / 5, ln(sigma) / ln 2, state / 8) for
 * n states; all inputs positive (state >= 0). */
int tps_ws_features(int n, const double *mass_ratio, const double *v0, const double *sigma,
                    const int *state, float *X_host);
/* Network outputs out[B][rank (px + py)] for features X[B][4] (device FP32); bf16 = 1 uses
 * the BF16 weights.  Asynchronous on stream. */
int tps_ws_forward(tps_ws *ws, const float *X_dev, int B, int bf16, float *out_dev,
                   cudaStream_t stream);
/* Forward + backward for a batch: mean loss (host, nullable) and dL/dparams kept in the
 * model for tps_ws_adam_step (also copied to grad_host[nparam] if not null).  Synchronous
 * when loss_host or grad_host is given. */
int tps_ws_loss_grad(tps_ws *ws, const float *X_dev, const float *T_dev, int B,
                     double *loss_host, float *grad_host, cudaStream_t stream);
/* One Adam step (Kingma & Ba) with the gradient of the last tps_ws_loss_grad call. */
int tps_ws_adam_step(tps_ws *ws, float lr, float beta1, float beta2, float eps,
                     cudaStream_t stream);
/* Training targets: T[v] = Phi^T psi_v Chi (px x py, FP32) of k eigenvectors evecs[k][N]
 * (device, FP64, the context's full grid).  Needs 2 px <= n_x and py < n_y in 1D;
 * q_x < n_x1, n_x2 and q_y < n_y1, n_y2 in 2D (TPS_ERR_INVALID_ARG otherwise). */
int tps_ws_project(tps_ws *ws, tps_ctx *ctx, const double *evecs_dev, int k, float *T_dev,
                   cudaStream_t stream);
/* Predicted states on the context's full grid: x0[k][N] (device FP64) for features
 * X[k][4] (device FP32).  Unnormalised; the solver orthonormalises its start block. */
int tps_ws_predict(tps_ws *ws, tps_ctx *ctx, const float *X_dev, int k, double *x0_dev,
                   cudaStream_t stream);
/* tps_solve started from the model's prediction for states 0 .. k + guard - 1 of
 * (mass_ratio, v0, sigma) (guard from opts, default 2; the solver's first block then
 * spans every wanted pair); if that solve does not converge, the cold-started solver
 * runs instead (*used_warm = 0).  ws = NULL: the cold-started solver.  Same outputs and
 * errors as tps_solve. */
int tps_ws_solve(tps_ws *ws, tps_ctx *ctx, double mass_ratio, double v0, double sigma, int k,
                 int parity, double tol, int block, const tps_solver_opts *opts,
                 double *evals_host, double *evecs_dev, tps_stats *stats, int *used_warm,
                 cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TPS_H */
