// Small device kernels of the Jacobi-Davidson outer loop and of the GMRES
// correction solver (Sec. 4.1): Hessenberg bookkeeping with Givens rotations, the
// small triangular solve, projected-basis matrix updates.  One thread per system or
// per matrix entry; all sizes are tiny (<= 64).
#include "jd_kernels.h"
#include "pdl.cuh"

namespace tps {
namespace {

// Layout of the GMRES state for system i (steps = s):
//   Hb[i] : (s+1) x s column-major (ld s+1)   Hessenberg, rotated in place
//   cs[i], sn[i] : s rotations   g[i] : s+1   beta[i], done[i], mvalid[i], scale[i]

__global__ void k_gmres_init(int nsys, int s, const double *nrm2, double *beta, double *g,
                             double *Hb, int *done, int *mvalid, double *scale) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsys) return;
  const double b = sqrt(nrm2[i] > 0.0 ? nrm2[i] : 0.0);
  beta[i] = b;
  for (int l = 0; l <= s; ++l) g[i * (s + 1) + l] = 0.0;
  g[i * (s + 1)] = b;
  for (int e = 0; e < (s + 1) * s; ++e) Hb[(long long)i * (s + 1) * s + e] = 0.0;
  const bool ok = b > 1e-300;
  done[i] = ok ? 0 : 1;
  mvalid[i] = 0;
  scale[i] = ok ? -1.0 / b : 0.0;  // z_0 = -Kt^-1 r / beta
}

__global__ void k_hess_add(int nsys, int s, int j, const double *h, int ldh, double *Hb,
                           const int *done) {
  pdl_entry();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = e / (j + 1), l = e % (j + 1);
  if (i >= nsys) return;
  if (done[i]) return;
  Hb[(long long)i * (s + 1) * s + (long long)j * (s + 1) + l] += h[(long long)i * ldh + l];
}

__global__ void k_gmres_givens(int nsys, int s, int j, const double *nrm2, double *Hb,
                               double *cs, double *sn, double *g, const double *beta, int *done,
                               int *mvalid, double *scale, double tol) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsys) return;
  if (done[i]) {
    scale[i] = 0.0;
    return;
  }
  double *H = Hb + (long long)i * (s + 1) * s + (long long)j * (s + 1);
  double *c = cs + i * s, *sv = sn + i * s, *gi = g + i * (s + 1);
  const double hnext = sqrt(nrm2[i] > 0.0 ? nrm2[i] : 0.0);
  H[j + 1] = hnext;
  for (int l = 0; l < j; ++l) {  // previous rotations
    const double a = H[l], b = H[l + 1];
    H[l] = c[l] * a + sv[l] * b;
    H[l + 1] = -sv[l] * a + c[l] * b;
  }
  const double a = H[j], b = H[j + 1];
  const double r = hypot(a, b);
  double cc = 1.0, ss = 0.0;
  if (r > 0.0) {
    cc = a / r;
    ss = b / r;
  }
  c[j] = cc;
  sv[j] = ss;
  H[j] = r;
  H[j + 1] = 0.0;
  gi[j + 1] = -ss * gi[j];
  gi[j] = cc * gi[j];
  if (r > 0.0) mvalid[i] = j + 1;
  const bool breakdown = !(hnext > 1e-14 * r) || !(r > 0.0);
  const bool conv = fabs(gi[j + 1]) <= tol * beta[i];
  if (breakdown || conv) {
    done[i] = 1;
    scale[i] = 0.0;
  } else {
    scale[i] = 1.0 / hnext;
  }
}

__global__ void k_gmres_solve(int nsys, int s, const double *Hb, const double *g,
                              const int *mvalid, double *y) {
  pdl_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsys) return;
  const double *H = Hb + (long long)i * (s + 1) * s;
  const double *gi = g + i * (s + 1);
  double *yi = y + i * s;
  const int m = mvalid[i];
  for (int l = m; l < s; ++l) yi[l] = 0.0;
  for (int l = m - 1; l >= 0; --l) {
    double v = gi[l];
    for (int k = l + 1; k < m; ++k) v -= H[(long long)k * (s + 1) + l] * yi[k];
    const double d = H[(long long)l * (s + 1) + l];
    yi[l] = d != 0.0 ? v / d : 0.0;
  }
}

// G[m0+a, m0+b] block symmetrised and mirrored: G[m0+b][c] = G[c][m0+b] for c < m0.
__global__ void k_mirror_block(double *G, int ldg, int m0, int bn) {
  pdl_entry();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int tot = (m0 + bn) * bn;
  if (e >= tot) return;
  const int col = m0 + e % bn;  // new column
  const int row = e / bn;       // 0 .. m0+bn-1
  if (row < m0) {
    G[(long long)row * ldg + col] = G[(long long)col * ldg + row];
  } else if (row < col) {
    const double a = G[(long long)col * ldg + row], b = G[(long long)row * ldg + col];
    const double v = 0.5 * (a + b);
    G[(long long)col * ldg + row] = v;
    G[(long long)row * ldg + col] = v;
  }
}

__global__ void k_set_diag(double *G, int ldg, const double *d, int m) {
  pdl_entry();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  const int i = e % m, j = e / m;
  G[(long long)j * ldg + i] = (i == j) ? d[i] : 0.0;
}

// dst[0:mk, 0:mk] = src[off:off+mk, off:off+mk] (column-major, leading dimensions lds, ldd)
__global__ void k_copy_block(const double *src, int lds, int off, double *dst, int ldd, int mk) {
  pdl_entry();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= mk * mk) return;
  const int i = e % mk, j = e / mk;
  dst[(long long)j * ldd + i] = src[(long long)(j + off) * lds + (i + off)];
}

__global__ void k_copy_small(const double *src, double *dst, int n) {
  pdl_entry();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) dst[e] = src[e];
}

__global__ void k_sqrt_div(const double *nrm2, double *out, int n, double div) {
  pdl_entry();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = sqrt(nrm2[e] > 0.0 ? nrm2[e] : 0.0) / div;
}

// C (m x n) = alpha * A (m x k) * B (k x n) + beta * C, column-major, tiny sizes
__global__ void k_small_gemm(int m, int n, int k, double alpha, const double *A, int lda,
                             const double *B, int ldb, double beta, double *C, int ldc) {
  pdl_entry();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * n) return;
  const int i = e % m, j = e / m;
  double v = 0.0;
  for (int l = 0; l < k; ++l) v += A[(long long)l * lda + i] * B[(long long)j * ldb + l];
  double *c = C + (long long)j * ldc + i;
  *c = (beta == 0.0) ? alpha * v : alpha * v + beta * *c;
}

inline unsigned nb(long long n, int t = 128) { return (unsigned)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

}  // namespace

void launch_gmres_init(int nsys, int s, const double *nrm2, GmresState &st, cudaStream_t str) {
  count_launch();
  launch_pdl(k_gmres_init, nb(nsys), 128, 0, str, nsys, s, nrm2, st.beta, st.g, st.Hb, st.done,
             st.mvalid,
                                           st.scale);
}
void launch_hess_add(int nsys, int s, int j, const double *h, int ldh, GmresState &st,
                     cudaStream_t str) {
  count_launch();
  launch_pdl(k_hess_add, nb((long long)nsys * (j + 1)), 128, 0, str, nsys, s, j, h, ldh, st.Hb,
             st.done);
}
void launch_gmres_givens(int nsys, int s, int j, const double *nrm2, GmresState &st, double tol,
                         cudaStream_t str) {
  count_launch();
  launch_pdl(k_gmres_givens, nb(nsys), 128, 0, str, nsys, s, j, nrm2, st.Hb, st.cs, st.sn, st.g,
             st.beta,
                                             st.done, st.mvalid, st.scale, tol);
}
void launch_gmres_solve(int nsys, int s, GmresState &st, cudaStream_t str) {
  count_launch();
  launch_pdl(k_gmres_solve, nb(nsys), 128, 0, str, nsys, s, st.Hb, st.g, st.mvalid, st.y);
}
// A column of the new block that the Cholesky-QR dropped (keep0 == 0) is zero, so its row
// and column of G are zero: its diagonal entry is raised to twice the largest |G_ii| of the
// first m0 + bn, which puts that spurious Ritz value above the wanted ones.
__global__ void k_mark_dropped(double *G, int ldg, int m0, int bn, const int *keep0) {
  pdl_entry();
  __shared__ double mx;
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < m0 + bn; ++i) a = fmax(a, fabs(G[(long long)i * ldg + i]));
    mx = a;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < bn; j += blockDim.x)
    if (!keep0[j]) G[(long long)(m0 + j) * ldg + (m0 + j)] = 2.0 * mx + 1.0;
}

// Convergence of the first k pairs (squared residual norms nrm2 <= thresh2), counted
// iterations, and the condition of the enclosing graph loop: go on while not converged and
// under the iteration cap.  state[0] = converged, state[1] = iterations.
__global__ void k_conv_check(const double *nrm2, int k, double thresh2, int *state, int max_iter,
                             cudaGraphConditionalHandle loop, int set_loop) {
  pdl_entry();
  if (threadIdx.x != 0) return;
  int conv = 1;
  for (int i = 0; i < k; ++i) conv = conv && nrm2[i] <= thresh2;
  state[0] = conv;
  state[1] += 1;
  if (set_loop) cudaGraphSetConditional(loop, (!conv && state[1] < max_iter) ? 1u : 0u);
}

// Residual columns of pairs already converged (nrm2 <= thresh2) are set to zero, so their
// corrections are zero (and dropped by the orthonormalisation) instead of noise directions.
__global__ void k_zero_converged(double *R, long long nrows, const double *nrm2, int k,
                                 double thresh2) {
  pdl_entry();
  const long long total = (long long)k * nrows;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    if (nrm2[e / nrows] <= thresh2) R[e] = 0.0;
}

// The preconditioner's shift from the lowest unconverged Ritz value theta: below the kinetic
// spectrum (bottom lam_min), at the mirror image of theta when theta lies above it:
// shift = lam_min - max(|theta - lam_min|, 1e-8 hnorm).
__global__ void k_shift_update(const double *theta, const double *nrm2, int k, double thresh2,
                               double lam_min, double hnorm, double *shift) {
  pdl_entry();
  if (threadIdx.x != 0) return;
  int i = 0;
  while (i < k - 1 && nrm2[i] <= thresh2) ++i;
  *shift = lam_min - fmax(fabs(theta[i] - lam_min), 1e-8 * hnorm);
}

namespace {

// Normal deviates for random start blocks, counter-based (a block depends on the seed and
// its counter only): the uniform u_i in (0, 1) is the top 24 bits of
// splitmix64(seed * 0x2545F4914F6CDD1D + i) plus 1/2, times 2^-24 (splitmix64: Steele, Lea &
// Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), and each pair
// (u_e, u_e+1) gives two deviates by the Box-Muller transform, in FP32 (a start block needs
// no more than random directions).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}
__device__ __forceinline__ float uniform01(uint64_t seed, uint64_t i) {
  return ((float)(splitmix64(seed * 0x2545F4914F6CDD1DULL + i) >> 40) + 0.5f) * (1.f / 16777216.f);
}
__global__ void k_fill_normal(double *dst, long long n, uint64_t seed, uint64_t offset) {
  pdl_entry();
  for (long long e = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x); e < n;
       e += 2LL * gridDim.x * blockDim.x) {
    const float u1 = uniform01(seed, offset + (uint64_t)e);
    const float u2 = uniform01(seed, offset + (uint64_t)e + 1);
    const float r = sqrtf(-2.f * logf(u1));
    float sn, cs;
    sincospif(2.f * u2, &sn, &cs);
    dst[e] = (double)(r * cs);
    if (e + 1 < n) dst[e + 1] = (double)(r * sn);
  }
}

}  // namespace

void launch_fill_normal(double *dst, long long n, uint64_t seed, uint64_t offset,
                        cudaStream_t str) {
  if (n <= 0) return;
  count_launch();
  long long blocks = (n / 2 + 256) / 256;
  if (blocks > 152LL * 8) blocks = 152LL * 8;
  launch_pdl(k_fill_normal, (unsigned)blocks, 256, 0, str, dst, n, seed, offset);
}

void launch_zero_converged(double *R, long long nrows, const double *nrm2, int k, double thresh2,
                           cudaStream_t str) {
  count_launch();
  long long blocks = ((long long)k * nrows + 255) / 256;
  if (blocks > 152LL * 8) blocks = 152LL * 8;
  launch_pdl(k_zero_converged, (unsigned)blocks, 256, 0, str, R, nrows, nrm2, k, thresh2);
}

void launch_shift_update(const double *theta, const double *nrm2, int k, double thresh2,
                         double lam_min, double hnorm, double *shift, cudaStream_t str) {
  count_launch();
  launch_pdl(k_shift_update, 1, 32, 0, str, theta, nrm2, k, thresh2, lam_min, hnorm, shift);
}

void launch_mark_dropped(double *G, int ldg, int m0, int bn, const int *keep0, cudaStream_t str) {
  count_launch();
  launch_pdl(k_mark_dropped, 1, 32, 0, str, G, ldg, m0, bn, keep0);
}

void launch_conv_check(const double *nrm2, int k, double thresh2, int *state, int max_iter,
                       cudaGraphConditionalHandle loop, int set_loop, cudaStream_t str) {
  count_launch();
  launch_pdl(k_conv_check, 1, 32, 0, str, nrm2, k, thresh2, state, max_iter, loop, set_loop);
}

void launch_mirror_block(double *G, int ldg, int m0, int bn, cudaStream_t str) {
  count_launch();
  launch_pdl(k_mirror_block, nb((long long)(m0 + bn) * bn), 128, 0, str, G, ldg, m0, bn);
}
void launch_set_diag(double *G, int ldg, const double *d, int m, cudaStream_t str) {
  count_launch();
  launch_pdl(k_set_diag, nb((long long)m * m), 128, 0, str, G, ldg, d, m);
}
void launch_copy_block(const double *src, int lds, int off, double *dst, int ldd, int mk,
                       cudaStream_t str) {
  count_launch();
  launch_pdl(k_copy_block, nb((long long)mk * mk), 128, 0, str, src, lds, off, dst, ldd, mk);
}
void launch_copy_small(const double *src, double *dst, int n, cudaStream_t str) {
  count_launch();
  launch_pdl(k_copy_small, nb(n), 128, 0, str, src, dst, n);
}
void launch_sqrt_div(const double *nrm2, double *out, int n, double div, cudaStream_t str) {
  count_launch();
  launch_pdl(k_sqrt_div, nb(n), 128, 0, str, nrm2, out, n, div);
}
void launch_small_gemm(int m, int n, int k, double alpha, const double *A, int lda, const double *B,
                       int ldb, double beta, double *C, int ldc, cudaStream_t str) {
  if (m <= 0 || n <= 0) return;
  count_launch();
  launch_pdl(k_small_gemm, nb((long long)m * n), 128, 0, str, m, n, k, alpha, A, lda, B, ldb, beta,
             C, ldc);
}

}  // namespace tps
