// FP64 block kernels for the Jacobi-Davidson steps of Sec. 4.1: tall-skinny Gram
// matrices and block updates (orthogonalisation, Rayleigh-Ritz projection, Ritz
// vectors, restarts, Arnoldi), the small dense Cholesky/Givens work on one CTA, and
// elementwise helpers (the small eigensolver is in rr_eigh.cu).  Everything stays on the device; the host only
// reads a few scalars per outer iteration to steer the loop.
#include <cstring>
#include <mutex>
#include <utility>

#include "pdl.cuh"
#include "tps_internal.h"

namespace tps {
namespace {

constexpr int GT = 256;  // threads of the Gram / update kernels

// -------------------------------- Gram ---------------------------------------
// G_s = A_s^T B_s in one launch.  CTA (c, s, pb) sums the BP x BQ block pb over the rows of
// chunk c into partial[s][pb][c][BP BQ]; the last CTA of a block to finish (ticket counter,
// after a memory fence) adds the chunks in chunk order -- the same order every call, so
// the result is deterministic -- writes the block into G and re-arms the counter.  The
// register tile fits the shape (16 x 1, 8 x 2, 4 x 4 and smaller), so narrow products do
// not pay for FMAs on padding; trans = 1 stores the transposed block (the launcher swaps
// the operands when p < q).  T = float: FP32 products and partial sums on the FP64 data
// (the low-precision variant; the chunk sums are added in FP64).
//
// Warp reduction of V = BP BQ values by recursive halving: at offset o each lane keeps
// half of its values and adds the other half of its partner's, so a lane spends V - 1 +
// (5 - log2 V) FP64 adds instead of 5 V -- FP64 instructions are the scarce resource on
// GB300.  Afterwards lane l holds the sum of value index sum_k bit(l, 4-k) V / 2^(k+1).
template <int V, typename T>
__device__ __forceinline__ void warp_halving_sum(T (&v)[V]) {
  const int lane = threadIdx.x & 31;
  int n = V;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if (n > 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < V / 2; ++i) {
        if (i < n / 2) {
          const T send = up ? v[i] : v[i + n / 2];
          const T keep = up ? v[i + n / 2] : v[i];
          v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
      }
      n >>= 1;
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    }
  }
}

template <int V>
__device__ __forceinline__ int halving_index(int lane) {
  int idx = 0, w = V / 2;
#pragma unroll
  for (int o = 16; o > 0 && w > 0; o >>= 1, w >>= 1) idx += (lane & o) ? w : 0;
  return idx;
}

template <int V>
__device__ __forceinline__ bool halving_writer(int lane) {  // one lane per value index
  int used = 0;
#pragma unroll
  for (int w = V / 2; w > 0; w >>= 1) ++used;  // offsets 16 .. 2^(5-used) carry the index
  return (lane & ((1 << (5 - used)) - 1)) == 0;
}

template <typename T, int BP, int BQ>
__global__ void __launch_bounds__(GT)
k_gram(const double *__restrict__ A, long long lda, long long bsa, int p,
       const double *__restrict__ B, long long ldb, long long bsb, int q, long long nrows,
       int nchunk, double *__restrict__ partial, unsigned *__restrict__ count,
       double *__restrict__ G, int ldg, long long bsg, int trans, const int *__restrict__ need) {
  pdl_entry();
  constexpr int V = BP * BQ;
  if (need && *need == 0) return;  // conditional product (decided on the device)
  const int c = blockIdx.x, s = blockIdx.y, pb = blockIdx.z;
  const int qb = (q + BQ - 1) / BQ;
  const int npb = ((p + BP - 1) / BP) * qb;
  const int i0 = (pb / qb) * BP, j0 = (pb % qb) * BQ;
  const double *As = A + s * bsa;
  const double *Bs = B + s * bsb;
  const long long rows_per = (nrows + nchunk - 1) / nchunk;
  const long long r0 = (long long)c * rows_per;
  const long long r1 = r0 + rows_per < nrows ? r0 + rows_per : nrows;
  T acc[V];
#pragma unroll
  for (int k = 0; k < V; ++k) acc[k] = T(0);
  // two rows per iteration: all of their loads are issued before the first FMA waits
  long long r = r0 + threadIdx.x;
  for (; r + GT < r1; r += 2 * GT) {
    T a[2][BP], b[2][BQ];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int i = 0; i < BP; ++i)
        a[h][i] = (i0 + i < p) ? (T)As[(long long)(i0 + i) * lda + r + h * GT] : T(0);
#pragma unroll
      for (int j = 0; j < BQ; ++j)
        b[h][j] = (j0 + j < q) ? (T)Bs[(long long)(j0 + j) * ldb + r + h * GT] : T(0);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int i = 0; i < BP; ++i)
#pragma unroll
        for (int j = 0; j < BQ; ++j) acc[i * BQ + j] = fma(a[h][i], b[h][j], acc[i * BQ + j]);
  }
  if (r < r1) {
    T a[BP], b[BQ];
#pragma unroll
    for (int i = 0; i < BP; ++i)
      a[i] = (i0 + i < p) ? (T)As[(long long)(i0 + i) * lda + r] : T(0);
#pragma unroll
    for (int j = 0; j < BQ; ++j)
      b[j] = (j0 + j < q) ? (T)Bs[(long long)(j0 + j) * ldb + r] : T(0);
#pragma unroll
    for (int i = 0; i < BP; ++i)
#pragma unroll
      for (int j = 0; j < BQ; ++j) acc[i * BQ + j] = fma(a[i], b[j], acc[i * BQ + j]);
  }
  warp_halving_sum<V>(acc);
  __shared__ T red[GT / 32][V];
  __shared__ unsigned ticket;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (halving_writer<V>(lane)) red[warp][halving_index<V>(lane)] = acc[0];
  __syncthreads();
  const long long blk = (long long)s * npb + pb;
  if (threadIdx.x < V) {
    T v = T(0);
    for (int w = 0; w < GT / 32; ++w) v += red[w][threadIdx.x];
    partial[(blk * nchunk + c) * V + threadIdx.x] = (double)v;
    __threadfence();  // this chunk's sums are visible before the ticket is taken
  }
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(&count[blk], 1u);
  __syncthreads();
  if (ticket != (unsigned)(nchunk - 1)) return;
  // last CTA of the block: every other chunk's partial sums are in memory
  if (threadIdx.x < V) {
    __threadfence();
    const double *src = partial + blk * nchunk * V + threadIdx.x;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    int cc = 0;
    for (; cc + 4 <= nchunk; cc += 4) {
      v0 += __ldcg(src + (long long)(cc + 0) * V);
      v1 += __ldcg(src + (long long)(cc + 1) * V);
      v2 += __ldcg(src + (long long)(cc + 2) * V);
      v3 += __ldcg(src + (long long)(cc + 3) * V);
    }
    for (; cc < nchunk; ++cc) v0 += __ldcg(src + (long long)cc * V);
    const double v = (v0 + v1) + (v2 + v3);
    const int i = i0 + threadIdx.x / BQ, j = j0 + threadIdx.x % BQ;
    if (i < p && j < q) {
      if (trans)
        G[s * bsg + (long long)i * ldg + j] = v;
      else
        G[s * bsg + (long long)j * ldg + i] = v;
    }
  }
  if (threadIdx.x == 0) count[blk] = 0u;  // re-armed for the next call on this stream
}

int gram_chunks(long long nrows, int batch, int npb) {
  const long long want = (2LL * 152 + (long long)batch * npb - 1) / ((long long)batch * npb);
  const long long maxc = (nrows + 1023) / 1024;
  long long c = want < maxc ? want : maxc;
  if (c < 1) c = 1;
  if (c > 1024) c = 1024;
  return (int)c;
}

// ------------------------------- update --------------------------------------
// C_s[:, j0:j0+BQ] = beta*C_s + alpha * A_s Y_s[:, j0:j0+BQ]; BQ fits q (1, 2, 4 or 8), so
// narrow updates do not pay for FMAs on padding columns, and a column block reads A once.
// T = float: FP32 products and sums on the FP64 data (the low-precision variant), the beta
// combination in FP64.  A grid of at most one wave of CTAs strides over the rows, two
// rows and four columns of A per thread in flight (a CTA per 256 rows spent most of its
// life loading Y).
template <typename T, int BQ>
__global__ void __launch_bounds__(GT)
k_update(const double *__restrict__ A, long long lda, long long bsa, int p,
         const double *__restrict__ Y, int ldy, long long bsy, int q, double alpha, double beta,
         double *__restrict__ C, long long ldc, long long bsc, long long nrows,
         const int *__restrict__ need) {
  pdl_entry();
  if (need && *need == 0) return;  // conditional product (decided on the device)
  const int s = blockIdx.y;
  const int j0 = blockIdx.z * BQ;
  __shared__ T Ys[64][BQ];
  for (int e = threadIdx.x; e < p * BQ; e += GT) {
    const int i = e / BQ, j = e % BQ;
    Ys[i][j] = (j0 + j < q) ? (T)(alpha * Y[s * bsy + (long long)(j0 + j) * ldy + i]) : T(0);
  }
  __syncthreads();
  const double *As = A + s * bsa;
  double *Cs = C + s * bsc;
  const long long stride = (long long)gridDim.x * GT;
  for (long long r0 = (long long)blockIdx.x * GT + threadIdx.x; r0 < nrows; r0 += 2 * stride) {
    const long long r1 = r0 + stride;
    const bool v1 = r1 < nrows;
    T acc0[BQ], acc1[BQ];
#pragma unroll
    for (int j = 0; j < BQ; ++j) acc0[j] = acc1[j] = T(0);
    int i = 0;
    for (; i + 4 <= p; i += 4) {
      T a0[4], a1[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a0[u] = (T)As[(long long)(i + u) * lda + r0];
        a1[u] = v1 ? (T)As[(long long)(i + u) * lda + r1] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int j = 0; j < BQ; ++j) {
          acc0[j] = fma(a0[u], Ys[i + u][j], acc0[j]);
          acc1[j] = fma(a1[u], Ys[i + u][j], acc1[j]);
        }
    }
    for (; i < p; ++i) {
      const T a0 = (T)As[(long long)i * lda + r0];
      const T a1 = v1 ? (T)As[(long long)i * lda + r1] : T(0);
#pragma unroll
      for (int j = 0; j < BQ; ++j) {
        acc0[j] = fma(a0, Ys[i][j], acc0[j]);
        acc1[j] = fma(a1, Ys[i][j], acc1[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < BQ; ++j) {
      if (j0 + j >= q) break;
      double *dst = Cs + (long long)(j0 + j) * ldc;
      dst[r0] = (beta == 0.0) ? (double)acc0[j] : fma(beta, dst[r0], (double)acc0[j]);
      if (v1) dst[r1] = (beta == 0.0) ? (double)acc1[j] : fma(beta, dst[r1], (double)acc1[j]);
    }
  }
}

// ------------------------------ Cholesky QR ----------------------------------
// 1/sqrt(d) for a normal d > 0 to FP64 accuracy without the FP64 square root and divide
// (each ~0.33 us of dependent latency on GB300): d = ds 4^h with ds in [1, 4), an FP32
// estimate of 1/sqrt(ds) and two FP64 Newton steps y <- y (3 - ds y^2) / 2 (2^-23 -> 2^-45
// -> rounding), then scaled by 2^-h.
__device__ __forceinline__ double rsqrt64(double d) {
  const long long bits = __double_as_longlong(d);
  const int e = (int)((bits >> 52) & 0x7ff) - 1023;
  const int h = e >> 1;  // floor(e / 2)
  const double ds = __longlong_as_double(bits - ((long long)(2 * h) << 52));
  double y = (double)rsqrtf((float)ds);
  y = y * (1.5 - 0.5 * ds * y * y);
  y = y * (1.5 - 0.5 * ds * y * y);
  return __longlong_as_double(__double_as_longlong(y) - ((long long)h << 52));
}

// Cholesky G = R^T R (R upper) of the b x b Gram matrix (b <= 32, one warp), dropping
// columns whose pivot falls below tol_rel^2 ref[j]; then Rinv by back substitution, a
// column per lane.  Pivots use rsqrt64 and every division is a multiplication by it.
__global__ void k_chol_inv(const double *__restrict__ G, int b, const double *__restrict__ ref,
                           double tol_rel, double *__restrict__ Rinv, int *__restrict__ keep) {
  pdl_entry();
  __shared__ double R[32][33];
  __shared__ double inv[32];
  __shared__ int kp[32];
  const int tid = threadIdx.x;
  for (int e = tid; e < b * b; e += blockDim.x) {
    const int i = e % b, j = e / b;
    R[i][j] = (i <= j) ? G[(long long)j * b + i] : 0.0;
  }
  __syncwarp();
  for (int j = 0; j < b; ++j) {
    if (tid == 0) {
      double d = R[j][j];
      for (int k = 0; k < j; ++k) d -= R[k][j] * R[k][j];
      const double rj = ref ? ref[j] : G[(long long)j * b + j];
      const int ok = (d > tol_rel * tol_rel * rj) && (d > 0.0) && (d > 1e-300);
      kp[j] = ok;
      if (ok) {
        const double y = rsqrt64(d);
        inv[j] = y;
        R[j][j] = d * y;
      } else {
        inv[j] = 0.0;
        R[j][j] = 0.0;
      }
    }
    __syncwarp();
    const int i = tid;
    if (i > j && i < b) {
      if (kp[j]) {
        double v = R[j][i];
        for (int k = 0; k < j; ++k) v -= R[k][j] * R[k][i];
        R[j][i] = v * inv[j];
      } else {
        R[j][i] = 0.0;  // the dropped column's row of R is zero
      }
    }
    __syncwarp();
  }
  // Rinv column c by back substitution (dropped rows/columns are zero)
  if (tid < b) {
    const int c = tid;
    double x[32];
    for (int i = 0; i < b; ++i) x[i] = 0.0;
    if (kp[c]) {
      for (int i = c; i >= 0; --i) {
        if (!kp[i]) {
          x[i] = 0.0;
          continue;
        }
        double v = (i == c) ? 1.0 : 0.0;
        for (int k = i + 1; k <= c; ++k) v -= R[i][k] * x[k];
        x[i] = v * inv[i];
      }
    }
    for (int i = 0; i < b; ++i) Rinv[(long long)c * b + i] = x[i];
    keep[c] = kp[c];
  }
}

// --------------------------- SPD inverse (small) ------------------------------
// Minv = M^-1 by Cholesky M = L L^T in place in Minv (lower), then L^-1, then L^-T L^-1;
// reciprocal pivots by rsqrt64, no FP64 division.
__global__ void k_spd_inverse(const double *__restrict__ M, int q, double *__restrict__ W) {
  pdl_entry();
  const int tid = threadIdx.x, nt = blockDim.x;
  extern __shared__ double sm[];
  double *Lm = sm;           // q x q, column-major
  double *Li = sm + q * q;   // q x q
  double *dinv = Li + q * q; // 1 / L[j][j]
  for (int e = tid; e < q * q; e += nt) {
    const int i = e % q, j = e / q;
    Lm[e] = 0.5 * (M[(long long)j * q + i] + M[(long long)i * q + j]);
    Li[e] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < q; ++j) {
    if (tid == 0) {
      double d = Lm[j * q + j];
      for (int k = 0; k < j; ++k) d -= Lm[k * q + j] * Lm[k * q + j];
      const double y = rsqrt64(d > 1e-300 ? d : 1e-300);
      dinv[j] = y;
      Lm[j * q + j] = (d > 1e-300 ? d : 1e-300) * y;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < q; i += nt) {
      double v = Lm[j * q + i];
      for (int k = 0; k < j; ++k) v -= Lm[k * q + i] * Lm[k * q + j];
      Lm[j * q + i] = v * dinv[j];
    }
    __syncthreads();
  }
  // Li = L^-1 column by column (forward substitution), one thread per column
  for (int c = tid; c < q; c += nt) {
    for (int i = c; i < q; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) v -= Lm[k * q + i] * Li[c * q + k];
      Li[c * q + i] = v * dinv[i];
    }
  }
  __syncthreads();
  // W = Li^T Li
  for (int e = tid; e < q * q; e += nt) {
    const int i = e % q, j = e / q;
    double v = 0.0;
    const int k0 = i > j ? i : j;
    for (int k = k0; k < q; ++k) v += Li[i * q + k] * Li[j * q + k];
    W[(long long)j * q + i] = v;
  }
}

// ------------------------------ elementwise ----------------------------------
// Eq. definition_potential on the 1D grid: V[i][j] = -v0 (f(|y_j - x_i/2|/sigma) +
// f(|y_j + x_i/2|/sigma)), f = exp(-xi^2) (shape 0) or (1 + xi^2)^-3 (shape 1), with
// x_i = -L_x + i 2L_x/n_x; also the FP32 copy.
__global__ void k_pair_potential_1d(int nx, int ny, double Lx, double Ly, int shape, double v0,
                                    double sigma, double *__restrict__ V, float *__restrict__ Vf) {
  pdl_entry();
  const long long total = (long long)nx * ny;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / ny), j = (int)(e % ny);
    const double x = -Lx + i * (2.0 * Lx / nx), y = -Ly + j * (2.0 * Ly / ny);
    const double a = fabs(y - 0.5 * x) / sigma, b = fabs(y + 0.5 * x) / sigma;
    double fa, fb;
    if (shape == 0) {
      fa = exp(-a * a);
      fb = exp(-b * b);
    } else {
      const double ta = 1.0 + a * a, tb = 1.0 + b * b;
      fa = 1.0 / (ta * ta * ta);
      fb = 1.0 / (tb * tb * tb);
    }
    const double v = -v0 * (fa + fb);
    V[e] = v;
    Vf[e] = (float)v;
  }
}

__global__ void k_axpby_cols(int ncols, long long nrows, double alpha, const double *X,
                             long long ldx, double beta, double *Y, long long ldy) {
  pdl_entry();
  const long long total = (long long)ncols * nrows;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / nrows, r = e % nrows;
    double *y = Y + c * ldy + r;
    const double xv = alpha * X[c * ldx + r];
    *y = (beta == 0.0) ? xv : fma(beta, *y, xv);
  }
}

__global__ void k_scale_cols(int ncols, long long nrows, const double *X, long long ldx,
                             const double *scale, int invert, double *Y, long long ldy) {
  pdl_entry();
  const long long total = (long long)ncols * nrows;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / nrows, r = e % nrows;
    double f = scale[c];
    if (invert) f = (f > 1e-300 || f < -1e-300) ? 1.0 / f : 0.0;
    Y[c * ldy + r] = X[c * ldx + r] * f;
  }
}

__global__ void k_residual(int ncols, long long nrows, const double *HX, const double *X,
                           const double *theta, double *R) {
  pdl_entry();
  const long long total = (long long)ncols * nrows;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / nrows;
    R[e] = fma(-theta[c], X[e], HX[e]);
  }
}

// Parity-reduced coordinates of the 1D grid (mode 0 = x folded by x -> -x):
//  even: u_i = sqrt(w_i) * (P_i + P_{n-i}) / 2, i = 0..n/2, w = (1, 2, .., 2, 1)
//  odd:  u_i = sqrt(2) * (P_i - P_{n-i}) / 2,   i = 1..n/2-1
__global__ void k_sector_restrict(int parity, int nx, int ny, int ncols, const double *full,
                                  double *red) {
  pdl_entry();
  const int nr = parity == TPS_X_EVEN ? nx / 2 + 1 : nx / 2 - 1;
  const long long Nf = (long long)nx * ny, Nr = (long long)nr * ny;
  const long long total = (long long)ncols * Nr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / Nr, rem = e % Nr;
    const int ir = (int)(rem / ny), j = (int)(rem % ny);
    const double *P = full + c * Nf;
    double v;
    if (parity == TPS_X_EVEN) {
      const int i = ir;
      if (i == 0 || i == nx / 2)
        v = P[(long long)i * ny + j];
      else
        v = sqrt(2.0) * 0.5 * (P[(long long)i * ny + j] + P[(long long)(nx - i) * ny + j]);
    } else {
      const int i = ir + 1;
      v = sqrt(2.0) * 0.5 * (P[(long long)i * ny + j] - P[(long long)(nx - i) * ny + j]);
    }
    red[c * Nr + rem] = v;
  }
}

__global__ void k_sector_expand(int parity, int nx, int ny, int ncols, const double *red,
                                double *full) {
  pdl_entry();
  const int nr = parity == TPS_X_EVEN ? nx / 2 + 1 : nx / 2 - 1;
  const long long Nf = (long long)nx * ny, Nr = (long long)nr * ny;
  const long long total = (long long)ncols * Nf;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / Nf, rem = e % Nf;
    const int i = (int)(rem / ny), j = (int)(rem % ny);
    const double *u = red + c * Nr;
    double v;
    if (parity == TPS_X_EVEN) {
      const int ir = i <= nx / 2 ? i : nx - i;
      const double w = (ir == 0 || ir == nx / 2) ? 1.0 : sqrt(0.5);
      v = w * u[(long long)ir * ny + j];
    } else {
      if (i == 0 || i == nx / 2) {
        v = 0.0;
      } else {
        const int ir = i < nx / 2 ? i : nx - i;
        const double sg = i < nx / 2 ? 1.0 : -1.0;
        v = sg * sqrt(0.5) * u[(long long)(ir - 1) * ny + j];
      }
    }
    full[c * Nf + rem] = v;
  }
}

// sign fix: one CTA per column, argmax |x| (lowest index on ties), flip if negative.
// |x| is compared through its bit pattern (sign cleared): for IEEE doubles that order is
// the numeric one, and integer compares avoid the slow FP64 pipe.
// Sign convention for returned eigenvectors: the entry of largest magnitude (the first
// such index on ties) is made positive.  Chunk c of column j records its largest |x| (bit
// pattern), the index, and that entry's sign in part[j][c]; k_sign_apply combines the
// chunks of a column in chunk order and negates its slice of the column if needed (the
// signs travel with the partials, so no block reads an entry another may be negating).
__global__ void k_sign_partial(long long nrows, const double *__restrict__ X, int nchunk,
                               unsigned long long *__restrict__ part) {
  pdl_entry();
  const int c = blockIdx.x, j = blockIdx.y;
  const double *x = X + (long long)j * nrows;
  const long long per = (nrows + nchunk - 1) / nchunk;
  const long long r0 = (long long)c * per, r1 = r0 + per < nrows ? r0 + per : nrows;
  unsigned long long best = 0;
  long long bi = r0 < nrows ? r0 : 0;
  int neg = 0;
  for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x[r]);
    const unsigned long long a = u & 0x7fffffffffffffffULL;
    if (a > best) {
      best = a;
      bi = r;
      neg = (int)(u >> 63);
    }
  }
  __shared__ unsigned long long sb[256];
  __shared__ long long si[256];
  __shared__ int sn[256];
  sb[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  sn[threadIdx.x] = neg;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const unsigned long long a = sb[threadIdx.x + o];
      const long long ai = si[threadIdx.x + o];
      if (a > sb[threadIdx.x] || (a == sb[threadIdx.x] && ai < si[threadIdx.x])) {
        sb[threadIdx.x] = a;
        si[threadIdx.x] = ai;
        sn[threadIdx.x] = sn[threadIdx.x + o];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    unsigned long long *pp = part + ((long long)j * nchunk + c) * 2;
    pp[0] = sb[0];
    pp[1] = ((unsigned long long)si[0] << 1) | (unsigned long long)sn[0];
  }
}

__global__ void k_sign_apply(long long nrows, double *__restrict__ X, int nchunk,
                             const unsigned long long *__restrict__ part) {
  pdl_entry();
  const int j = blockIdx.y;
  __shared__ int neg;
  if (threadIdx.x == 0) {
    unsigned long long best = 0, tag = 0;
    bool have = false;
    for (int c = 0; c < nchunk; ++c) {  // chunk order = index order: ties keep the first
      const unsigned long long a = part[((long long)j * nchunk + c) * 2];
      const unsigned long long t = part[((long long)j * nchunk + c) * 2 + 1];
      if (!have || a > best) {
        best = a;
        tag = t;
        have = true;
      }
    }
    neg = (int)(tag & 1ull);
  }
  __syncthreads();
  if (!neg) return;
  double *x = X + (long long)j * nrows;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nrows;
       r += (long long)gridDim.x * blockDim.x)
    x[r] = -x[r];
}

unsigned grid_for(long long total, int threads = 256) {
  long long b = (total + threads - 1) / threads;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

long long gram_scratch_doubles(int p, int q, int batch) {
  const int npb = ((p + 3) / 4) * ((q + 3) / 4);
  return (long long)batch * npb * 1024 * 16;
}

void launch_gram(const double *A, long long lda, long long bsa, int p, const double *B,
                 long long ldb, long long bsb, int q, long long nrows, double *G, int ldg,
                 long long bsg, int batch, GramScratch &scr, cudaStream_t s, const int *need,
                 bool low) {
  if (p <= 0 || q <= 0 || batch <= 0) return;
  int trans = 0;
  if (p < q) {  // G^T = B^T A: the wider operand along the register tile's long side
    std::swap(A, B);
    std::swap(lda, ldb);
    std::swap(bsa, bsb);
    std::swap(p, q);
    trans = 1;
  }
  auto pow2 = [](int x, int lo, int hi) {
    int v = lo;
    while (v < x && v < hi) v <<= 1;
    return v;
  };
  const int BQ = q == 1 ? 1 : (q == 2 ? 2 : 4);
  const int BP = BQ == 1 ? pow2(p, 1, 16) : (BQ == 2 ? pow2(p, 2, 8) : 4);
  const int npb = ((p + BP - 1) / BP) * ((q + BQ - 1) / BQ);
  const int V = BP * BQ;
  int nchunk = gram_chunks(nrows, batch, npb);
  // partial sums fit the scratch; sized with 16 values per block at least, so that
  // batch * npb also stays below the ticket count (one per 16 doubles of capacity)
  const long long cap = scr.capacity / ((long long)batch * npb * (V > 16 ? V : 16));
  if (nchunk > cap) nchunk = (int)(cap > 0 ? cap : 1);
  dim3 grid(nchunk, batch, npb);
  count_launch();
#define TPS_GRAM(bp, bq)                                                                      \
  (low ? launch_pdl(k_gram<float, bp, bq>, grid, GT, 0, s, A, lda, bsa, p, B, ldb, bsb, q, nrows,  \
                    nchunk,                                                                        \
                                                   scr.partial, scr.count, G, ldg, bsg, trans,     \
                                                   need)                                           \
       : launch_pdl(k_gram<double, bp, bq>, grid, GT, 0, s, A, lda, bsa, p, B, ldb, bsb, q, nrows, \
                    nchunk,                                                                        \
                                                    scr.partial, scr.count, G, ldg, bsg, trans,    \
                                                    need))
  if (BQ == 4)
    TPS_GRAM(4, 4);
  else if (BQ == 2)
    BP == 2 ? TPS_GRAM(2, 2) : (BP == 4 ? TPS_GRAM(4, 2) : TPS_GRAM(8, 2));
  else
    BP == 1 ? TPS_GRAM(1, 1)
            : (BP == 2 ? TPS_GRAM(2, 1)
                       : (BP == 4 ? TPS_GRAM(4, 1) : (BP == 8 ? TPS_GRAM(8, 1) : TPS_GRAM(16, 1))));
#undef TPS_GRAM
}

// Resident CTAs per SM of k_update<T, BQ> (queried once per instantiation).
int update_occupancy(bool low, int BQ) {
  static int occ[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  static std::once_flag once;
  std::call_once(once, [] {
    const void *fn[2][4] = {{(const void *)k_update<double, 1>, (const void *)k_update<double, 2>,
                             (const void *)k_update<double, 4>, (const void *)k_update<double, 8>},
                            {(const void *)k_update<float, 1>, (const void *)k_update<float, 2>,
                             (const void *)k_update<float, 4>, (const void *)k_update<float, 8>}};
    for (int t = 0; t < 2; ++t)
      for (int b = 0; b < 4; ++b) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn[t][b], GT, 0) != cudaSuccess)
          n = 2;
        occ[t][b] = n < 1 ? 1 : n;
      }
  });
  return occ[low ? 1 : 0][BQ == 1 ? 0 : (BQ == 2 ? 1 : (BQ == 4 ? 2 : 3))];
}

void launch_update(const double *A, long long lda, long long bsa, int p, const double *Y, int ldy,
                   long long bsy, int q, double alpha, double beta, double *C, long long ldc,
                   long long bsc, long long nrows, int batch, cudaStream_t s, const int *need,
                   bool low) {
  if (q <= 0 || batch <= 0 || nrows <= 0) return;
  if (p <= 0) {  // C = beta * C
    for (int b = 0; b < batch; ++b) {
      count_launch();
      launch_pdl(k_axpby_cols, grid_for((long long)q * nrows), 256, 0, s, q, nrows, 0.0,
                 C + b * bsc, ldc,
                                                                beta, C + b * bsc, ldc);
    }
    return;
  }
  const int BQ = q > 4 ? 8 : (q > 2 ? 4 : q);
  const int zb = (q + BQ - 1) / BQ;
  // one wave: as many CTAs as fit on the SMs at once (over all systems and column blocks),
  // each striding over the rows
  const int occ = update_occupancy(low, BQ);
  long long gx = (nrows + 2 * GT - 1) / (2 * GT);
  const long long wave = std::max(1LL, 152LL * occ / ((long long)batch * zb));
  if (gx > 8 * wave) gx = wave;  // short inputs keep a CTA per 512 rows
  // p is processed in slabs of 64 rows of Y; the first slab applies beta
  for (int i0 = 0; i0 < p; i0 += 64) {
    const int pp = p - i0 < 64 ? p - i0 : 64;
    dim3 grid((unsigned)gx, batch, zb);
    const double bt = i0 == 0 ? beta : 1.0;
    const double *Ai = A + (long long)i0 * lda;
    count_launch();
#define TPS_UPD(T, bq)                                                                       \
  launch_pdl(k_update<T, bq>, grid, GT, 0, s, Ai, lda, bsa, pp, Y + i0, ldy, bsy, q, alpha, bt, C, \
             ldc,                                                                                  \
                                      bsc, nrows, need)
    if (low)
      BQ == 8 ? TPS_UPD(float, 8) : (BQ == 4 ? TPS_UPD(float, 4) : (BQ == 2 ? TPS_UPD(float, 2) : TPS_UPD(float, 1)));
    else
      BQ == 8 ? TPS_UPD(double, 8) : (BQ == 4 ? TPS_UPD(double, 4) : (BQ == 2 ? TPS_UPD(double, 2) : TPS_UPD(double, 1)));
#undef TPS_UPD
  }
}

// out[c] = sum_r A[c][r]^2 for ncols columns (ld lda): one pass, one FMA per element.
// Block (chunk, c) sums its rows into partial[c][chunk]; the last block of a column (ticket
// after a fence) adds the chunks in order and re-arms the ticket.
__global__ void __launch_bounds__(GT)
k_col_norms2(const double *__restrict__ A, long long lda, long long nrows, int nchunk,
             double *__restrict__ partial, unsigned *__restrict__ count, double *__restrict__ out) {
  pdl_entry();
  const int chunk = blockIdx.x, c = blockIdx.y;
  const long long rows_per = (nrows + nchunk - 1) / nchunk;
  const long long r0 = (long long)chunk * rows_per;
  const long long r1 = r0 + rows_per < nrows ? r0 + rows_per : nrows;
  const double *a = A + (long long)c * lda;
  // four independent loads in flight per thread
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  long long r = r0 + threadIdx.x;
  for (; r + 3 * GT < r1; r += 4 * GT) {
    const double x0 = a[r], x1 = a[r + GT], x2 = a[r + 2 * GT], x3 = a[r + 3 * GT];
    s0 = fma(x0, x0, s0);
    s1 = fma(x1, x1, s1);
    s2 = fma(x2, x2, s2);
    s3 = fma(x3, x3, s3);
  }
  for (; r < r1; r += GT) s0 = fma(a[r], a[r], s0);
  double v = (s0 + s1) + (s2 + s3);
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __shared__ double red[GT / 32];
  __shared__ unsigned ticket;
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < GT / 32; ++w) t += red[w];
    partial[(long long)c * nchunk + chunk] = t;
    __threadfence();
    ticket = atomicAdd(&count[c], 1u);
  }
  __syncthreads();
  if (threadIdx.x >= 32 || ticket != (unsigned)(nchunk - 1)) return;
  // the last CTA of the column: warp 0 adds the chunks' sums, all loads issued at once,
  // in a fixed order (lane-strided sums, then a fixed shuffle tree)
  __threadfence();
  const double *pc = partial + (long long)c * nchunk;
  double t = 0.0;
  for (int k = threadIdx.x; k < nchunk; k += 32) t += __ldcg(pc + k);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (threadIdx.x == 0) {
    out[c] = t;
    count[c] = 0u;
  }
}

__global__ void k_dgks_flag(const double *__restrict__ before, const double *__restrict__ after,
                            int ncols, int *__restrict__ need, int *__restrict__ stat) {
  pdl_entry();
  if (threadIdx.x != 0) return;
  int n = 0;
  for (int j = 0; j < ncols; ++j) n |= after[j] < 0.5 * before[j];
  *need = n;
  if (stat) {
    stat[0] += n;
    stat[1] += 1;
  }
}

void launch_col_norms2(const double *A, long long lda, int ncols, long long nrows, double *out,
                       GramScratch &scr, cudaStream_t s) {
  if (ncols <= 0) return;
  long long nchunk = (2LL * 152 + ncols - 1) / ncols;
  const long long maxc = (nrows + 2047) / 2048;
  if (nchunk > maxc) nchunk = maxc;
  if (nchunk > scr.capacity / ncols) nchunk = scr.capacity / ncols;
  if (nchunk < 1) nchunk = 1;
  count_launch();
  launch_pdl(k_col_norms2, dim3((unsigned)nchunk, ncols), GT, 0, s, A, lda, nrows, (int)nchunk,
                                                           scr.partial, scr.count, out);
}

void launch_dgks_flag(const double *before, const double *after, int ncols, int *need,
                      int *stat, cudaStream_t s) {
  count_launch();
  launch_pdl(k_dgks_flag, 1, 32, 0, s, before, after, ncols, need, stat);
}

void launch_pair_potential_1d(int nx, int ny, double Lx, double Ly, int shape, double v0,
                              double sigma, double *V, float *Vf, cudaStream_t s) {
  count_launch();
  launch_pdl(k_pair_potential_1d, grid_for((long long)nx * ny), 256, 0, s, nx, ny, Lx, Ly, shape,
             v0,
                                                                   sigma, V, Vf);
}

void launch_chol_inv(const double *G, int b, const double *ref, double tol_rel, double *Rinv,
                     int *keep, cudaStream_t s) {
  count_launch();
  launch_pdl(k_chol_inv, 1, 32, 0, s, G, b, ref, tol_rel, Rinv, keep);
}

void launch_spd_inverse(const double *M, int q, double *Minv, cudaStream_t s) {
  const size_t smem = (2 * (size_t)q * q + q) * sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_spd_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (2 * 96 * 96 + 96) * (int)sizeof(double));
    attr = true;
  }
  count_launch();
  launch_pdl(k_spd_inverse, 1, 128, smem, s, M, q, Minv);
}

void launch_axpby_cols(int ncols, long long nrows, double alpha, const double *X, long long ldx,
                       double beta, double *Y, long long ldy, cudaStream_t s) {
  if (ncols <= 0 || nrows <= 0) return;
  count_launch();
  launch_pdl(k_axpby_cols, grid_for((long long)ncols * nrows), 256, 0, s, ncols, nrows, alpha, X,
             ldx,
                                                                   beta, Y, ldy);
}

void launch_scale_cols(int ncols, long long nrows, const double *X, long long ldx,
                       const double *scale, int invert, double *Y, long long ldy, cudaStream_t s) {
  if (ncols <= 0 || nrows <= 0) return;
  count_launch();
  launch_pdl(k_scale_cols, grid_for((long long)ncols * nrows), 256, 0, s, ncols, nrows, X, ldx,
             scale,
                                                                   invert, Y, ldy);
}

void launch_residual(int ncols, long long nrows, const double *HX, const double *X,
                     const double *theta, double *R, cudaStream_t s) {
  if (ncols <= 0) return;
  count_launch();
  launch_pdl(k_residual, grid_for((long long)ncols * nrows), 256, 0, s, ncols, nrows, HX, X, theta,
             R);
}

void launch_sector_restrict(int parity, int nx, int ny, int ncols, const double *full,
                            double *red, cudaStream_t s) {
  const int nr = parity == TPS_X_EVEN ? nx / 2 + 1 : nx / 2 - 1;
  count_launch();
  launch_pdl(k_sector_restrict, grid_for((long long)ncols * nr * ny), 256, 0, s, parity, nx, ny,
             ncols,
                                                                         full, red);
}

void launch_sector_expand(int parity, int nx, int ny, int ncols, const double *red,
                          double *full, cudaStream_t s) {
  count_launch();
  launch_pdl(k_sector_expand, grid_for((long long)ncols * nx * ny), 256, 0, s, parity, nx, ny,
             ncols, red,
                                                                       full);
}

namespace {
__global__ void k_mirror_restrict(int sg, int nx, int ny, int ncols, const double *full,
                                  double *red) {
  pdl_entry();
  const int nr = nx / 2;
  const long long Nf = (long long)nx * ny, Nr = (long long)nr * ny;
  const long long total = (long long)ncols * Nr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / Nr, rem = e % Nr;
    const int i = (int)(rem / ny), j = (int)(rem % ny);
    const double *P = full + c * Nf;
    red[c * Nr + rem] =
        sqrt(0.5) * (P[(long long)i * ny + j] + sg * P[(long long)(nx - 1 - i) * ny + j]);
  }
}
__global__ void k_mirror_expand(int sg, int nx, int ny, int ncols, const double *red,
                                double *full) {
  pdl_entry();
  const int nr = nx / 2;
  const long long Nf = (long long)nx * ny, Nr = (long long)nr * ny;
  const long long total = (long long)ncols * Nf;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / Nf, rem = e % Nf;
    const int i = (int)(rem / ny), j = (int)(rem % ny);
    const int ir = i < nr ? i : nx - 1 - i;
    const double w = i < nr ? sqrt(0.5) : sg * sqrt(0.5);
    full[c * Nf + rem] = w * red[c * Nr + (long long)ir * ny + j];
  }
}
}  // namespace

void launch_mirror_restrict(int parity, int nx, int ny, int ncols, const double *full,
                            double *red, cudaStream_t s) {
  count_launch();
  launch_pdl(k_mirror_restrict, grid_for((long long)ncols * (nx / 2) * ny), 256, 0, s,
      parity == TPS_X_EVEN ? 1 : -1, nx, ny, ncols, full, red);
}

void launch_mirror_expand(int parity, int nx, int ny, int ncols, const double *red,
                          double *full, cudaStream_t s) {
  count_launch();
  launch_pdl(k_mirror_expand, grid_for((long long)ncols * nx * ny), 256, 0, s,
      parity == TPS_X_EVEN ? 1 : -1, nx, ny, ncols, red, full);
}

void launch_fix_sign(int ncols, long long nrows, double *X, GramScratch &scr, cudaStream_t s) {
  if (ncols <= 0 || nrows <= 0) return;
  long long nchunk = (4LL * 152 + ncols - 1) / ncols;
  const long long maxc = (nrows + 4095) / 4096;
  if (nchunk > maxc) nchunk = maxc;
  if (nchunk > scr.capacity / (2LL * ncols)) nchunk = scr.capacity / (2LL * ncols);
  if (nchunk < 1) nchunk = 1;
  unsigned long long *part = reinterpret_cast<unsigned long long *>(scr.partial);
  count_launch();
  launch_pdl(k_sign_partial, dim3((unsigned)nchunk, ncols), 256, 0, s, nrows, X, (int)nchunk, part);
  long long blocks = (nrows + 255) / 256;
  if (blocks > 152LL * 4 / ncols + 1) blocks = 152LL * 4 / ncols + 1;
  count_launch();
  launch_pdl(k_sign_apply, dim3((unsigned)blocks, ncols), 256, 0, s, nrows, X, (int)nchunk, part);
}

}  // namespace tps
