// Internal declarations of the tps library: device operator description,
// kernel launchers and the context.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tps.h"

namespace tps {

// Every kernel launch of the library is counted (reported by tps_solve's stats).
extern std::atomic<long long> g_kernel_launches;
inline void count_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
// GEMM tile autotuning switch (tps_set_autotune).
extern std::atomic<int> g_autotune;
inline bool autotune_enabled() { return g_autotune.load(std::memory_order_relaxed) != 0; }

// ---------------------------------------------------------------------------
// A discretised Kronecker-sum operator resident on the device:
//   H = sum_k (I x .. x K_k x .. x I) + diag(V),  K_k = a_k D2_k (dense n_k x n_k),
// with the orthonormal eigendecomposition K_k = S_k diag(lam_k) S_k^T used by the
// preconditioner.  nmodes = 2 (1D) or 4 (2D); the vector layout is C order over
// (n_0, .., n_{nmodes-1}).  The same struct describes the full grid and the
// parity-reduced operators of the solver (mode 0 folded, Sec. 5.1).
// ---------------------------------------------------------------------------
struct DevOperator {
  int nmodes = 0;
  int n[4] = {0, 0, 0, 0};
  long long N = 0;
  double *K[4] = {nullptr, nullptr, nullptr, nullptr};   // row-major n x n
  double *KT[4] = {nullptr, nullptr, nullptr, nullptr};  // K^T (equal to K for symmetric D2)
  double *S[4] = {nullptr, nullptr, nullptr, nullptr};   // row-major, columns = eigenvectors
  double *ST[4] = {nullptr, nullptr, nullptr, nullptr};  // S^T
  double *lam[4] = {nullptr, nullptr, nullptr, nullptr}; // eigenvalues of K_k
  float *Sf[4] = {nullptr, nullptr, nullptr, nullptr};   // FP32 copies for the FP32 paths
  float *STf[4] = {nullptr, nullptr, nullptr, nullptr};
  float *lamf[4] = {nullptr, nullptr, nullptr, nullptr};
  float *Kf[4] = {nullptr, nullptr, nullptr, nullptr};
  float *KTf[4] = {nullptr, nullptr, nullptr, nullptr};
  float *Vf = nullptr;
  double *V = nullptr;                                   // [N]
  std::vector<double> lam_h[4];                          // host copies (singularity test)
  std::vector<double> lam_rest;  // sorted sums of the eigenvalues of modes 1.. (singularity
                                 // test; empty when there are more than 2^22 of them)
  double lam_min_sum = 0.0, lam_max_sum = 0.0;
  bool owns = true;
  // tensor-core (BF16 digit slice) form of the mode matrices, built on first use
  mutable struct TcOperator *tc = nullptr;
  // padded FP32 eigenbases for the TF32 tensor-core preconditioner, built on first use
  mutable struct TfOperator *tf = nullptr;
};

// Workspace for one operator application (preconditioner intermediates).
struct ApplyWorkspace {
  double *t0 = nullptr, *t1 = nullptr;
  long long capacity = 0;  // doubles per buffer
};

// ------------------------------- launchers ----------------------------------
// out[v] = (H - theta_v) psi[v], theta_v = theta_dev ? theta_dev[v] : theta.
void launch_apply_h(const DevOperator &op, const double *psi, double *out, int nvec,
                    const double *theta_dev, double theta, cudaStream_t s);
// out[v] = (T - sigma)^-1 r[v] by fast diagonalisation (needs 2 * nvec * N workspace).
void launch_apply_prec(const DevOperator &op, const double *r, double *out, int nvec,
                       double sigma, ApplyWorkspace &ws, cudaStream_t s);
// out[v] = (H - theta_v) psi[v] with FP32 arithmetic (FP64 psi and out; psi is converted
// once into the workspace, which must hold nvec * N floats).
void launch_apply_h_f32(const DevOperator &op, const double *psi, double *out, int nvec,
                        const double *theta_dev, double theta, ApplyWorkspace &ws,
                        cudaStream_t s);
// The same with FP32 arithmetic (FP64 r and out).
void launch_apply_prec_f32(const DevOperator &op, const double *r, double *out, int nvec,
                           double sigma, ApplyWorkspace &ws, cudaStream_t s);

// FP64-accurate 1D H-apply on the tensor cores (Ozaki digit splitting); builds op.tc on
// first use.  Asynchronous on s.
cudaError_t launch_apply_h_tc(const DevOperator &op, const double *psi, double *out, int nvec,
                              const double *theta_dev, double theta, cudaStream_t s);
cudaError_t ensure_tc_operator(const DevOperator &op, cudaStream_t s);
void free_tc_operator(struct TcOperator *t);
// TF32 tensor-core preconditioner: out[v] = (T - sigma)^-1 r[v] with the mode products
// in TF32 (four in 1D, eight in 2D; FP64 r and out; the FP32 intermediates use the
// workspace, which must hold tf_prec_workspace_floats / 2 doubles).  ensure_tf_operator
// builds op.tf (padded eigenbases, synchronous); the launcher returns TPS_ERR_INVALID_ARG
// without it.  tf_prec_supported: 1D, or 2D with every mode 4 .. 128 points, a multiple of 4.
bool tf_prec_supported(const DevOperator &op);
void free_tf_operator(struct TfOperator *t);
int ensure_tf_operator(const DevOperator &op);
long long tf_prec_workspace_floats(const DevOperator &op, int nvec);
// sigma_dev (nullable): the shift read on the device, in place of sigma.
int launch_apply_prec_tf32(const DevOperator &op, const double *r, double *out, int nvec,
                           double sigma, ApplyWorkspace &ws, cudaStream_t s,
                           const double *sigma_dev = nullptr);
int tf_operator_status(const DevOperator &op);
// Synchronously reads and clears the timed-out-wait flag of op's tensor-core kernels.
int tc_operator_status(const DevOperator &op);

// Skinny block kernels.  Column c of block X is X + c*ldx; batch s adds s*bsx.
struct GramScratch {
  double *partial = nullptr;
  long long capacity = 0;     // doubles
  unsigned *count = nullptr;  // per-block tickets of the one-launch Gram, zero between calls
  long long ncount = 0;
};
// G_s = A_s^T B_s (p x q, column-major ldg) for s < batch.  need (device, nullable): the
// product is skipped when *need == 0 (a decision taken by an earlier kernel).
// low: FP32 products and sums on the FP64 data (~1e-7 relative), for the correction
// equation, which is solved to 1e-3 and whose result is re-orthogonalised in FP64.
void launch_gram(const double *A, long long lda, long long bsa, int p, const double *B,
                 long long ldb, long long bsb, int q, long long nrows, double *G, int ldg,
                 long long bsg, int batch, GramScratch &scr, cudaStream_t s,
                 const int *need = nullptr, bool low = false);
// C_s = beta*C_s + alpha * A_s Y_s (Y column-major p x q, ldy, batch stride bsy); need as
// for launch_gram.
void launch_update(const double *A, long long lda, long long bsa, int p, const double *Y, int ldy,
                   long long bsy, int q, double alpha, double beta, double *C, long long ldc,
                   long long bsc, long long nrows, int batch, cudaStream_t s,
                   const int *need = nullptr, bool low = false);
// The same update, FP64-accurate, as digit-split BF16 products on the tensor cores
// (update_mma.cu); q any, p any (slabs of 64).
void launch_update_split(const double *A, long long lda, long long bsa, int p, const double *Y,
                         int ldy, long long bsy, int q, double alpha, double beta, double *C,
                         long long ldc, long long bsc, long long nrows, int batch, cudaStream_t s,
                         const int *need = nullptr);
// G = A^T B, FP64-accurate, as digit-split BF16 products on the tensor cores (gram_mma.cu),
// exponents per 64-row block; for batch 1, min(p, q) <= 8 and max(p, q) <= 64
// (gram_split_supported); need as for launch_gram.
bool gram_split_supported(int p, int q, int batch);
// the split is faster than the FMA pipe's Gram from p q >= 32 on (measured at 131,584 rows)
bool gram_split_pays(int p, int q);
// low: three digits per operand (23-bit truncation, FP32-quality products) for the
// correction equation, like launch_gram's low.
void launch_gram_split(const double *A, long long lda, int p, const double *B, long long ldb,
                       int q, long long nrows, double *G, int ldg, GramScratch &scr,
                       cudaStream_t s, const int *need = nullptr, bool low = false);
// Queries the split update's launch configuration for every slab width up front (before
// a stream capture).
void prewarm_update_split();
// Synchronously reads and clears the timed-out-wait flag of the staged split update
// (1 if a wait gave up since the last call, 0 if not, -1 if the flag cannot be read).
int update_split_status();
// Host: A = S diag(lam) S^-1 for a real n x n row-major A with a real spectrum (ascending
// lam, unit columns of S; Sinv nullable).  0 on success, 1 for a complex pair or no
// convergence, 2 for a singular S (host_eig.cpp).
int real_eig(int n, const double *A, double *lam, double *S, double *Sinv);
// Host: the k eigenvalues of smallest real part of a real n x n row-major A (real parts,
// ascending) and real unit eigenvectors Y (column c at Y + c ldy); imag_max (nullable) gets
// the largest |imaginary part| among them.  0 on success, 1 if the QR steps do not converge
// (host_eig.cpp).
int complex_eig_lowest(int n, const double *A, int k, double *lam, double *Y, int ldy,
                       double *imag_max);
// out[c] = squared 2-norm of column c (ld lda, nrows rows), c < ncols; uses scr.
void launch_col_norms2(const double *A, long long lda, int ncols, long long nrows, double *out,
                       GramScratch &scr, cudaStream_t s);
// *need = 1 if any column lost more than half its squared norm: after[j] < 0.5 before[j]
// (the DGKS criterion for a second Gram-Schmidt pass); also counts the decision in
// stat[0] (passes needed) and stat[1] (decisions), stat nullable.
void launch_dgks_flag(const double *before, const double *after, int ncols, int *need,
                      int *stat, cudaStream_t s);

// Small dense kernels (one CTA or one cluster each).
// Eigenpairs of the symmetric m x m G (ld ldg): theta ascending, Y column-major (ld ldy).
// mp > 0: the leading mp x mp block of G is unchanged since the previous call, whose
// outputs theta[:mp] and Y[:mp, :mp] are still in theta and Y; they seed the solve and are
// overwritten.  stat (device, nullable): adds sweeps, rounds with rotations and 1 to
// stat[0..2].  tol_abs: off-diagonal entries below max(4 eps |A|_F, tol_abs) are left.
// Arot (device, nullable, ld ldy): receives Y^T G Y (theta on its diagonal, the entries
// left below the threshold off it); with mp > 0 its leading block is read as the
// previous call's rotated matrix instead of diag(theta).
// This entry runs the FP64 cyclic Jacobi method.
void launch_jacobi_eigh(const double *G, int m, int ldg, double *theta, double *Y, int ldy,
                        cudaStream_t s, int mp = 0, int *stat = nullptr, double tol_abs = 0.0,
                        double *Arot = nullptr);
// The same contract by `method` (TPS_RR_MIXED: FP32 Jacobi + FP64 refinement, with the
// FP64 Jacobi inside the same launch when the refinement does not converge;
// TPS_RR_JACOBI64: FP64 Jacobi).  stat (nullable) needs 8 ints: [0..2] as above for the
// FP64 Jacobi, [3] mixed calls, [4] FP32 eigensolves, [5] refinement iterations, [6] groups of
// close eigenvalues rotated, [7] calls that fell back to the FP64 Jacobi.  refine_max:
// refinement iterations before the fallback (<= 0: 12).
void launch_rr_eigh(const double *G, int m, int ldg, double *theta, double *Y, int ldy,
                    cudaStream_t s, int mp, int *stat, double tol_abs, double *Arot, int method,
                    int refine_max = 0);
// Cholesky G = R^T R of the b x b Gram matrix (ld b); writes Rinv (upper, ld b) and
// keep[c] = 1 if column c has a pivot >= tol_rel * ref[c] (ref = squared column norms
// before projection, device, may be null), else 0 (column dropped, Rinv column zero).
void launch_chol_inv(const double *G, int b, const double *ref, double tol_rel, double *Rinv,
                     int *keep, cudaStream_t s);
// Minv = M^-1 for an SPD q x q matrix (column-major, ld q).
void launch_spd_inverse(const double *M, int q, double *Minv, cudaStream_t s);

// Elementwise helpers.
// The pair potential of Eq. definition_potential on the full 1D grid (FP64 and FP32 copies).
void launch_pair_potential_1d(int nx, int ny, double Lx, double Ly, int shape, double v0,
                              double sigma, double *V, float *Vf, cudaStream_t s);
void launch_axpby_cols(int ncols, long long nrows, double alpha, const double *X, long long ldx,
                       double beta, double *Y, long long ldy, cudaStream_t s);
// Y[:, c] = X[:, c] * scale[c] (scale device); safe in place.
void launch_scale_cols(int ncols, long long nrows, const double *X, long long ldx,
                       const double *scale, int invert, double *Y, long long ldy, cudaStream_t s);
// R[:, c] = HX[:, c] - theta[c] * X[:, c]
void launch_residual(int ncols, long long nrows, const double *HX, const double *X,
                     const double *theta, double *R, cudaStream_t s);
// expand/restrict between the full 1D grid and a parity-reduced one.
void launch_sector_restrict(int parity, int nx, int ny, int ncols, const double *full,
                            double *red, cudaStream_t s);
void launch_sector_expand(int parity, int nx, int ny, int ncols, const double *red,
                          double *full, cudaStream_t s);
// the same for the mirror-symmetric Chebyshev x grid (x_i = -x_{n-1-i}, no node at 0):
// u_i = (P_i +- P_{n-1-i}) / sqrt 2, i < n/2, for both sectors.
void launch_mirror_restrict(int parity, int nx, int ny, int ncols, const double *full,
                            double *red, cudaStream_t s);
void launch_mirror_expand(int parity, int nx, int ny, int ncols, const double *red,
                          double *full, cudaStream_t s);
// flip the sign of each column so that its entry of largest magnitude is positive.
void launch_fix_sign(int ncols, long long nrows, double *X, GramScratch &scr, cudaStream_t s);

// ------------------------------- context ------------------------------------
struct SolverWorkspace;

}  // namespace tps

struct tps_ctx {
  int device = 0;
  int dim = 1;
  bool have_masses = false, have_grid = false, have_V = false;
  double a[2] = {0, 0};  // kinetic coefficient of x and y
  int n[4] = {0, 0, 0, 0};
  double L[4] = {0, 0, 0, 0};
  int grid_kind = 0;                   // 0: Fourier grids (tps_set_grid); 1: mapped Chebyshev
                                       // roots (tps_set_grid_chebyshev, 1D)
  std::vector<double> pts[2];          // grid points of x and y (mapped Chebyshev grids)
  std::vector<double> V_host;          // potential on the full grid
  mutable double vmax = 0.0;           // max |V_host| (tps_get_info), valid if vmax_ok
  mutable bool vmax_ok = false;
  tps::DevOperator full;               // full grid operator
  tps::DevOperator sect[3];            // [TPS_X_EVEN], [TPS_X_ODD] parity-reduced 1D operators
  bool sect_ready[3] = {false, false, false};
  tps::ApplyWorkspace ws;
  tps::GramScratch gscr;
  tps::SolverWorkspace *sw = nullptr;
  std::string err;
};

namespace tps {
// Error helpers used by the API layer.
int set_error(tps_ctx *ctx, int code, const std::string &msg);
int cuda_error(tps_ctx *ctx, cudaError_t e, const char *where);
int ensure_apply_workspace(tps_ctx *ctx, long long doubles);
int ensure_gram_scratch(tps_ctx *ctx, long long doubles);
void free_operator(DevOperator &op);
// Build the parity-reduced 1D operator for TPS_X_EVEN / TPS_X_ODD.
int build_sector_operator(tps_ctx *ctx, int parity);
// The outer loop as one captured CUDA graph with a device-side convergence test (jd.cpp);
// TPS_ERR_NOT_CONVERGED when the caller should fall back to solve_impl.
int solve_graph_impl(tps_ctx *ctx, int k, int parity, double tol, const tps_solver_opts &opts,
                     double *evals_host, double *evecs_dev, tps_stats *stats,
                     cudaStream_t stream);
// The eigensolver for the non-symmetric H of the mapped Chebyshev grid (jd.cpp).
int solve_nonsym_impl(tps_ctx *ctx, int k, int parity, double tol, int block,
                      const tps_solver_opts *opts, double *evals_host, double *evecs_dev,
                      tps_stats *stats, cudaStream_t stream);
int solve_impl(tps_ctx *ctx, int k, int parity, double tol, int block, const double *x0,
               int n_x0, const tps_solver_opts *opts, double *evals_host, double *evecs_dev,
               tps_stats *stats, cudaStream_t stream);
void free_solver_workspace(tps_ctx *ctx);
long long gram_scratch_doubles(int p, int q, int batch);
// shift_dev (nullable): the preconditioner's shift read on the device (TF32 preconditioner
// only), in place of shift.
int correction_impl(tps_ctx *ctx, const DevOperator &op, const double *Qt, int nq,
                    const double *KQt_cached, int nq_cached, const double *R,
                    const double *theta, int nsys, int steps, int use_prec, double shift,
                    double inner_tol, double *T, int *h_applies, int *prec_applies,
                    cudaStream_t s, bool direction_only, bool low,
                    const double *shift_dev = nullptr);
}  // namespace tps

#define TPS_CUDA_TRY(ctx, expr)                                   \
  do {                                                            \
    cudaError_t _e = (expr);                                      \
    if (_e != cudaSuccess) return tps::cuda_error(ctx, _e, #expr); \
  } while (0)
