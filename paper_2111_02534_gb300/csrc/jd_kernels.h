// Launchers of the small Jacobi-Davidson / GMRES device kernels.
#pragma once

#include "tps_internal.h"

namespace tps {

struct GmresState {
  double *Hb = nullptr;     // [nsys][(s+1) * s]
  double *cs = nullptr;     // [nsys][s]
  double *sn = nullptr;     // [nsys][s]
  double *g = nullptr;      // [nsys][s+1]
  double *beta = nullptr;   // [nsys]
  double *scale = nullptr;  // [nsys]
  double *y = nullptr;      // [nsys][s]
  double *h = nullptr;      // [nsys][s+1] one Arnoldi column
  double *nrm2 = nullptr;   // [nsys]
  int *done = nullptr;      // [nsys]
  int *mvalid = nullptr;    // [nsys]
};

void launch_gmres_init(int nsys, int s, const double *nrm2, GmresState &st, cudaStream_t str);
void launch_hess_add(int nsys, int s, int j, const double *h, int ldh, GmresState &st,
                     cudaStream_t str);
void launch_gmres_givens(int nsys, int s, int j, const double *nrm2, GmresState &st, double tol,
                         cudaStream_t str);
void launch_gmres_solve(int nsys, int s, GmresState &st, cudaStream_t str);
void launch_mirror_block(double *G, int ldg, int m0, int bn, cudaStream_t str);
void launch_mark_dropped(double *G, int ldg, int m0, int bn, const int *keep0, cudaStream_t str);
void launch_zero_converged(double *R, long long nrows, const double *nrm2, int k, double thresh2,
                           cudaStream_t str);
void launch_shift_update(const double *theta, const double *nrm2, int k, double thresh2,
                         double lam_min, double hnorm, double *shift, cudaStream_t str);
void launch_conv_check(const double *nrm2, int k, double thresh2, int *state, int max_iter,
                       cudaGraphConditionalHandle loop, int set_loop, cudaStream_t str);
void launch_set_diag(double *G, int ldg, const double *d, int m, cudaStream_t str);
void launch_copy_block(const double *src, int lds, int off, double *dst, int ldd, int mk,
                       cudaStream_t str);
void launch_copy_small(const double *src, double *dst, int n, cudaStream_t str);
void launch_sqrt_div(const double *nrm2, double *out, int n, double div, cudaStream_t str);
// dst[0 .. n) = standard normal deviates i = offset .. offset + n - 1 of the seed's
// counter-based stream (random start blocks)
void launch_fill_normal(double *dst, long long n, uint64_t seed, uint64_t offset,
                        cudaStream_t str);
void launch_small_gemm(int m, int n, int k, double alpha, const double *A, int lda, const double *B,
                       int ldb, double beta, double *C, int ldc, cudaStream_t str);

}  // namespace tps
