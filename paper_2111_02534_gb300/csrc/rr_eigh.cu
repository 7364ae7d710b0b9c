// Rayleigh-Ritz eigensolver of Sec. 4.1: all eigenpairs of the small projected matrix
// G = V^T H V (m <= 64), ascending, on one thread-block cluster of 8 CTAs.
//
// Two methods:
//  * jacobi64 -- cyclic Jacobi in FP64 (round-robin parallel ordering).  Robust for any
//    spectrum, but a sweep is m - 1 dependent rounds, each a chain of FP64 instructions
//    and a cluster barrier; GB300 issues FP64 at a small fraction of its FP32 rate, so a
//    call at m = 32 costs about half a millisecond.
//  * k_rr_mixed (default) -- a FP32 eigensolver with O(m) dependent steps gives starting
//    vectors, and FP64 is spent on a few dense products instead of m - 1 rounds per sweep:
//      1. eig32 below (Householder tridiagonalisation, multisection, inverse iteration) on
//         A0 / ||A0||_F in FP32, replicated in every CTA (the same data and instructions
//         give the same result in each, so no cross-CTA traffic);
//      2. FP64 iterative refinement of the eigenvector matrix X (T. Ogita, K. Aishima,
//         "Iterative refinement for symmetric eigenvalue decomposition", Japan J. Indust.
//         Appl. Math. 35 (2018)): R = I - X^T X, S = X^T A0 X (symmetrised),
//         lambda_i = s_ii / (1 - r_ii), X <- X (I + E) with
//         E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) across groups of close
//         eigenvalues and E_ij = r_ij / 2 inside one; quadratically convergent.  A group
//         is a run of sorted lambda_i with gaps <= delta = 2 m (max|s_ij| + ||A0||_F max|r_ij|),
//         an upper bound of the authors' 2-norm expression.  The products are spread over
//         the cluster: CTA r owns rows (and columns) r R .. r R + R - 1, R = ceil(m / 8);
//      3. inside a group with off-diagonals above the threshold, the block predicted for
//         after the update, T_ij = s_ij + (lambda_i + lambda_j) r_ij / 2, T_ii = lambda_i,
//         is diagonalised by eig32 after shifting by one of its eigenvalue estimates and
//         scaling by its largest entry; two FP64 Newton-Schulz steps make
//         that rotation orthogonal to FP64 rounding, and X_J <- X_J W_J (the treatment of
//         clustered eigenvalues in the authors' follow-up, JJIAM 36 (2019));
//      4. the iteration stops when every off-diagonal of S is at most
//         thr = max(8.9e-16 ||A0||_F, tol_abs) and every entry of R at most 4 m 2^-53.
//         If it has not after refine_max iterations the same kernel runs jacobi64 on the
//         unchanged inputs, so the result never depends on the refinement converging.
//
// Warm start (mp > 0, both methods): the leading mp x mp block of G is the projection
// onto a basis whose Ritz pairs (Y[:mp, :mp], theta[:mp]) the previous call returned,
// and only the trailing columns are new.  The matrix diagonalised is A0 = Q0^T G Q0 with
// Q0 = diag(Y_prev, I): its leading block is the previous call's rotated matrix (Arot,
// else diag(theta)), and the coupling block Y_prev^T G_12 holds the previous Ritz
// vectors' residuals against the new columns.  The result is Q0 V.  theta, Y and Arot
// are read before they are written, so they may be updated in place.
#include <cooperative_groups.h>

#include <atomic>

#include "pdl.cuh"
#include "tps_internal.h"

namespace cg = cooperative_groups;

namespace tps {
namespace {

constexpr int JMAX = 64;
constexpr int JCL = 8;                 // CTAs per cluster
constexpr int JROWS = JMAX / JCL;      // rows per CTA at most
constexpr int JT = 256;                // threads per CTA
constexpr int JOUT = (JROWS * JMAX + JT - 1) / JT;  // output elements per thread
constexpr int LD = JMAX + 1;           // padded row length of the square work arrays

// symmetric part of G
__device__ __forceinline__ double g_sym(const double *G, int ldg, int r, int c) {
  return 0.5 * (G[(long long)c * ldg + r] + G[(long long)r * ldg + c]);
}

// Element (gi, j) of A0 = Q0^T G Q0 (see the warm start above).  The coupling entries
// are formed from the same terms in the same order for (gi, j) and (j, gi), so A0 is
// exactly symmetric.
__device__ double a0_entry(const double *G, int ldg, const double *theta, const double *Yp,
                           int ldy, int mp, const double *Arot, int gi, int j) {
  if (gi < mp && j < mp)
    return Arot ? 0.5 * (Arot[(long long)j * ldy + gi] + Arot[(long long)gi * ldy + j])
                : ((gi == j) ? theta[gi] : 0.0);
  double v = 0.0;
  if (gi < mp) {  // (Y_prev^T G)[gi][j] = sum_a Y[a][gi] G[a][j]
#pragma unroll 8
    for (int a = 0; a < mp; ++a) v = fma(Yp[(long long)gi * ldy + a], g_sym(G, ldg, a, j), v);
    return v;
  }
  if (j < mp) {  // (G Y_prev)[gi][j], the same terms in the same order
#pragma unroll 8
    for (int a = 0; a < mp; ++a) v = fma(Yp[(long long)j * ldy + a], g_sym(G, ldg, gi, a), v);
    return v;
  }
  return g_sym(G, ldg, gi, j);
}

// ------------------------------ FP64 cyclic Jacobi ----------------------------------
// Round-robin (tournament) ordering: each round rotates mm/2 disjoint pairs at once (Golub
// & Van Loan, symmetric Schur decomposition and the parallel ordering of the cyclic
// Jacobi method); A' = J^T A J is formed element by element from the two pairs an
// element's row and column belong to, V' = V J likewise.  CTA r owns a slab of rows of
// A and V and reads the partner rows it needs from the other CTAs' shared memory.  Every
// CTA computes the (identical) rotation parameters of a round itself, so one cluster
// barrier per round is the only cross-CTA synchronisation, and the exit decision of each
// sweep is CTA 0's, read by all.
struct JacobiSmem {
  double A[2][JROWS][LD];
  double Vv[2][JROWS][LD];
  double rc[JMAX], rs[JMAX];
  int partner[JMAX];
  double diag[JMAX];
  int perm[JMAX];
  int ipos[JMAX];
  double part[JT / 32];
  double norm_part;  // this CTA's squared Frobenius norm, read by the others
  int rotated[2];    // per sweep parity; CTA 0's flag decides for the cluster
  int act[JMAX];     // index rotates in this round
  int round_rot[2];  // any pair rotates in this round (by running round parity)
};

__device__ void jacobi64(JacobiSmem &sh, cg::cluster_group &cluster, const double *__restrict__ G,
                         int m, int ldg, double *theta, double *Yout, int ldy, int mp,
                         int *__restrict__ stat, double tol_abs, double *Arot) {
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  const int mm = (m + 1) & ~1;          // even number of players (m odd: one dummy)
  const int R = (mm + JCL - 1) / JCL;   // rows per CTA
  const int r0 = rank * R;
  // element (row, col) of A in buffer buf, wherever its row lives
  auto Aat = [&](int buf, int row, int col) -> double {
    const double *p = cluster.map_shared_rank(&sh.A[buf][row % R][col], (unsigned)(row / R));
    return *p;
  };
  double f = 0.0;
  for (int e = tid; e < R * mm; e += JT) {
    const int i = e / mm, j = e % mm, gi = r0 + i;
    double v = 0.0;
    if (gi < m && j < m) v = a0_entry(G, ldg, theta, Yout, ldy, mp, Arot, gi, j);
    sh.A[0][i][j] = v;
    sh.Vv[0][i][j] = (gi == j) ? 1.0 : 0.0;
    f += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
  if ((tid & 31) == 0) sh.part[tid >> 5] = f;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < JT / 32; ++w) t += sh.part[w];
    sh.norm_part = t;
    sh.round_rot[0] = sh.round_rot[1] = 0;
  }
  cluster.sync();
  double nrm2 = 0.0;
  for (int c = 0; c < JCL; ++c) nrm2 += *cluster.map_shared_rank(&sh.norm_part, (unsigned)c);
  const double normA = sqrt(nrm2);
  // entries below thr are left: the noise floor, or the caller's tolerance when the
  // eigenvectors are only needed to a given accuracy
  const double thr = fmax(8.9e-16 * normA, tol_abs);
  const double inv_norm = normA > 0.0 ? 1.0 / normA : 0.0;
  int cur = 0;
  long long rnd = 0;
  int sweeps = 0, rotating_rounds = 0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    ++sweeps;
    const int fl = sweep & 1;
    __syncthreads();
    if (tid == 0) sh.rotated[fl] = 0;
    __syncthreads();
    for (int r = 0; r < mm - 1; ++r, ++rnd) {
      cluster.sync();  // A[cur] complete in every CTA
      // pairs of this round (circle method): (mm-1, r), ((r+k) mod (mm-1), (r-k) mod (mm-1));
      // all pairs in one warp: FP64 work is paid per warp instruction
      if (tid < mm / 2) {
        const int k = tid;
        int pi, qi;
        if (k == 0) {
          pi = mm - 1;
          qi = r;
        } else {
          pi = (r + k) % (mm - 1);
          qi = (r - k + (mm - 1)) % (mm - 1);
        }
        const int p = pi < qi ? pi : qi, q = pi < qi ? qi : pi;
        double c = 1.0, sn = 0.0;
        if (q < m) {
          // the three loads go out together (one DSMEM round trip)
          const double apq = Aat(cur, p, q), app = Aat(cur, p, p), aqq = Aat(cur, q, q);
          // rotate unless a_pq is negligible relative to its diagonal pair or below the
          // rounding noise that rotations of the largest entries leave behind (4 eps
          // ||A||_F); chasing entries under that floor never terminates.  Squared forms:
          // an FP64 square root or division costs about ten FMAs' latency on this GPU.
          if (apq * apq > 1e-36 * fabs(app * aqq) && fabs(apq) > thr) {
            // t = tan(angle) zeroing a_pq: sign(d) a_pq / (|d| + sqrt(d^2 + a_pq^2)),
            // d = (a_qq - a_pp)/2, in FP32 on normA-scaled values; the rotation below is
            // orthogonal for any t, and a slightly inexact t leaves a_pq reduced by ~1e7
            const float df = (float)(0.5 * (aqq - app) * inv_norm);
            const float af = (float)(apq * inv_norm);
            const float tf = (df >= 0.f ? af : -af) / (fabsf(df) + sqrtf(df * df + af * af));
            const double t = (double)tf;
            // c = (1 + t^2)^(-1/2): FP32 estimate and two FP64 Newton steps (orthogonal to
            // FP64 rounding), s = t c
            const double u = 1.0 + t * t;
            double cc = (double)rsqrtf((float)u);
            cc = cc * (1.5 - 0.5 * u * cc * cc);
            cc = cc * (1.5 - 0.5 * u * cc * cc);
            c = cc;
            sn = t * cc;
            sh.rotated[fl] = 1;
            sh.round_rot[rnd & 1] = 1;
          }
        }
        sh.act[p] = sh.act[q] = (sn != 0.0);
        // column p of J = c e_p - s e_q ; column q of J = s e_p + c e_q
        sh.partner[p] = q;
        sh.partner[q] = p;
        sh.rc[p] = c;
        sh.rs[p] = -sn;
        sh.rc[q] = c;
        sh.rs[q] = sn;
      }
      __syncthreads();
      // a round without rotations changes nothing: keep the buffers.  Every CTA computed
      // the same parameters, so all of them take the same branch (and the barrier count
      // per round does not depend on it either way).  The other parity's flag is reset
      // here: its last readers passed the barrier above, its next writers come after the
      // next cluster barrier.
      const int any_rot = sh.round_rot[rnd & 1];
      if (tid == 0) sh.round_rot[(rnd + 1) & 1] = 0;
      if (!any_rot) continue;
      ++rotating_rounds;
      const int nxt = cur ^ 1;
      for (int e = tid; e < R * mm; e += JT) {
        const int i = e / mm, j = e % mm, gi = r0 + i;
        if (gi >= mm) continue;
        if (!sh.act[gi] && !sh.act[j]) {  // both rotations are the identity here
          sh.A[nxt][i][j] = sh.A[cur][i][j];
          sh.Vv[nxt][i][j] = sh.Vv[cur][i][j];
          continue;
        }
        const int pi = sh.partner[gi], pj = sh.partner[j];
        const double ci = sh.rc[gi], si = sh.rs[gi], cj = sh.rc[j], sj = sh.rs[j];
        // A'[i][j] = sum_{a in {i,pi}, b in {j,pj}} J[a][i] J[b][j] A[a][b]
        const double v = ci * (cj * sh.A[cur][i][j] + sj * sh.A[cur][i][pj]) +
                         si * (cj * Aat(cur, pi, j) + sj * Aat(cur, pi, pj));
        sh.A[nxt][i][j] = v;
        sh.Vv[nxt][i][j] = cj * sh.Vv[cur][i][j] + sj * sh.Vv[cur][i][pj];
      }
      cur = nxt;
    }
    // every CTA takes CTA 0's decision, so all of them run the same number of barriers;
    // CTA 0 resets the other parity's flag next sweep, so this read cannot race with it
    __syncthreads();
    cluster.sync();
    const int go = *cluster.map_shared_rank(&sh.rotated[fl], 0u);
    if (!go) break;
  }
  cluster.sync();  // final A and V complete everywhere
  if (stat && rank == 0 && tid == 0) {  // sweeps, rounds with rotations, calls
    atomicAdd(&stat[0], sweeps);
    atomicAdd(&stat[1], rotating_rounds);
    atomicAdd(&stat[2], 1);
  }
  for (int i = tid; i < m; i += JT) sh.diag[i] = Aat(cur, i, i);
  __syncthreads();
  // ascending order by rank (ties by index)
  for (int i = tid; i < m; i += JT) {
    int rk = 0;
    const double di = sh.diag[i];
    for (int j = 0; j < m; ++j) rk += (sh.diag[j] < di) || (sh.diag[j] == di && j < i);
    sh.perm[rk] = i;
  }
  __syncthreads();
  // the rotated matrix in sorted order: Arot[pos(c)][pos(r)] = A[r][c], pos = perm^-1.
  // Arot is read (warm start) before the first cluster barrier, so it may be updated here
  if (Arot) {
    for (int i = tid; i < m; i += JT) sh.ipos[sh.perm[i]] = i;
    __syncthreads();
    for (int e = tid; e < R * m; e += JT) {
      const int i = e / m, c = e % m, gi = r0 + i;
      if (gi < m) Arot[(long long)sh.ipos[c] * ldy + sh.ipos[gi]] = sh.A[cur][i][c];
    }
  }
  // Y[:, j] = (Q0 V)[:, perm[j]] for this CTA's rows, formed in registers first: with a
  // warm start every CTA reads the previous Y, which is overwritten in place
  double yv[JOUT];
#pragma unroll
  for (int t = 0; t < JOUT; ++t) {
    const int e = tid + t * JT;
    double v = 0.0;
    if (e < R * m) {
      const int i = e / m, j = e % m, gi = r0 + i;
      const int pj = sh.perm[j];
      if (gi < mp) {  // sum_a Y_prev[gi][a] V[a][pj]; row a of V lives in CTA a / R
#pragma unroll 8
        for (int a = 0; a < mp; ++a)
          v = fma(Yout[(long long)a * ldy + gi],
                  *cluster.map_shared_rank(&sh.Vv[cur][a % R][pj], (unsigned)(a / R)), v);
      } else if (gi < m) {
        v = sh.Vv[cur][i][pj];
      }
    }
    yv[t] = v;
  }
  cluster.sync();  // every CTA is done reading the previous Y
#pragma unroll
  for (int t = 0; t < JOUT; ++t) {
    const int e = tid + t * JT;
    if (e < R * m) {
      const int i = e / m, j = e % m, gi = r0 + i;
      if (gi < m) Yout[(long long)j * ldy + gi] = yv[t];
    }
  }
  if (rank == 0)
    for (int j = tid; j < m; j += JT) theta[j] = sh.diag[sh.perm[j]];
  cluster.sync();  // keep this CTA's shared memory alive until the others are done
}

__global__ void __cluster_dims__(JCL, 1, 1) __launch_bounds__(JT)
k_jacobi(const double *__restrict__ G, int m, int ldg, double *theta, double *Yout, int ldy,
         int mp, int *__restrict__ stat, double tol_abs, double *Arot) {
  pdl_entry();
  __shared__ JacobiSmem sh;
  cg::cluster_group cluster = cg::this_cluster();
  jacobi64(sh, cluster, G, m, ldg, theta, Yout, ldy, mp, stat, tol_abs, Arot);
}

// ------------------------- FP32 Jacobi + FP64 refinement ----------------------------
constexpr int kRefineMax = 12;  // default refinement iterations before the FP64 Jacobi

struct MixedSmem {
  float a[2][JMAX][JMAX + 1];  // FP32 solve: matrix and reflectors; inverse-iteration factors
  float v[JMAX][JMAX + 1];     //             eigenvectors
  double A0[JMAX][LD];         // A0, replicated
  double X[JMAX][LD];          // eigenvector estimate, replicated
  double F[JMAX][LD];          // the symmetrised S, replicated; scratch for group rotations
  double P[JMAX][LD];          // group blocks T, then their rotations
  double W[JMAX][JROWS + 1];   // own columns of A0 X
  double S[JMAX][JROWS + 1];   // own columns of X^T A0 X    (read by the other CTAs)
  double R[JMAX][JROWS + 1];   // own columns of I - X^T X   (read by the other CTAs)
  double E[JMAX][JROWS + 1];   // own columns of the correction E
  double Xn[JMAX][JROWS + 1];  // own columns of the next X  (read by the other CTAs)
  double lam[JMAX];            // lambda_i
  double rd[JMAX];             // r_ii
  long long key[JMAX];         // order-preserving integer keys
  double dred[JT / 32];
  unsigned long long bred[JT / 32];
  double norm2;                // this CTA's share of ||A0||_F^2 (read by the others)
  unsigned long long rmax;     // this CTA's max |r_ij| as bits (read by the others)
  double nrmA, inv, delta;
  unsigned long long thr_bits, rall_bits, gmask;
  unsigned int cscale[JMAX];   // per group (first list entry): max |T - shift| (float bits)
  unsigned long long coff[JMAX];  // per group (first list entry): max off-diagonal |T|
  int owner[JMAX], loc[JMAX];  // CTA owning row / column i, and its index there
  int order[JMAX];             // indices by ascending lambda
  int ipos[JMAX];              // inverse of order
  int gfirst[JMAX], gsize[JMAX];  // per sorted position: first position and size of its group
  int ml[JMAX];                // sorted positions of the members of groups of two or more
  int mbeg[JMAX], mend[JMAX];  // per ml entry: range of its group in ml
  int flag[JMAX], cnt[JMAX];   // scratch flags and prefix counts
  int clist[JMAX];             // ml entries of the groups rotated
  int cbeg[JMAX], cend[JMAX];  // per clist entry: range of its group in clist
  float td[JMAX], te[JMAX], te2[JMAX], tbeta[JMAX], tp[JMAX], tlam[JMAX];  // FP32 solve
  float tlo, thi;
  unsigned long long tcmask, tsmask;
  int nm, nc;
  int solves32, groups_rot;
};
static_assert(sizeof(MixedSmem) <= 227 * 1024, "shared memory per CTA");

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
}

// order-preserving integer image of a (non-NaN) double
__device__ __forceinline__ long long order_key(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}

// max over the CTA, returned to every thread (integer operations only)
__device__ unsigned long long cta_max_u64(unsigned long long v, unsigned long long *red) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long r = red[0];
#pragma unroll
  for (int w = 1; w < JT / 32; ++w) r = red[w] > r ? red[w] : r;
  __syncthreads();
  return r;
}

// inclusive prefix count of flag[0..n-1] (n <= 64) into cnt, by warp 0
__device__ void warp0_prefix(const int *flag, int n, int *cnt) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const unsigned b0 = __ballot_sync(0xffffffffu, lane < n && flag[lane]);
  const unsigned b1 = __ballot_sync(0xffffffffu, lane + 32 < n && flag[lane + 32]);
  const unsigned le = 0xffffffffu >> (31 - lane);
  if (lane < n) cnt[lane] = __popc(b0 & le);
  if (lane + 32 < n) cnt[lane + 32] = __popc(b0) + __popc(b1 & le);
}

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP32 symmetric eigensolver for the starting vectors of the refinement, on one CTA (each
// CTA of the cluster runs it on the same data): sh.a[0][0:n][0:n] (symmetric, destroyed)
// -> sh.v[0:n][0:n], column j the eigenvector of the (j+1)-th smallest eigenvalue.
//  1. Householder tridiagonalisation T = Q^T A Q (Golub & Van Loan, Householder
//     tridiagonalisation): step k reflects A[k+1:, k] with H = I - beta v v^T, v stored in
//     A[k+1:, k]; three barriers per step, A22 v a row per thread.
//  2. T splits into independent segments where |e_i| <= u (|d_i| + |d_{i+1}|) (block-diagonal
//     input splits exactly); column j belongs to the segment holding index j and takes its
//     (j - start)-th eigenvalue: multisection, G threads per eigenvalue evaluating Sturm
//     counts (the signs of the LDL^T pivots of the segment minus x I) at G points per step.
//  3. eigenvectors of the segments by two steps of inverse iteration, one thread per
//     eigenvalue (LDL^T of T - lambda I with pivots kept above u ||T||), the vectors of
//     eigenvalues of one segment closer than 1e-4 ||T|| made orthonormal by modified
//     Gram-Schmidt after each step (LAPACK's stein does so below 1e-3), one warp per
//     such cluster.
//  4. back-transformation X = Q Z by the stored reflectors, a few threads per column and
//     no barrier.
// The refinement needs only well-conditioned FP32-quality vectors: close eigenvalues whose
// vectors this leaves mixed are separated by its group rotations.
__device__ void eig32(MixedSmem &sh, int n, int c0 = 0, int c1 = -1) {
  if (c1 < 0) c1 = n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float(*A)[JMAX + 1] = sh.a[0];
  // 1. tridiagonalisation; each step: every warp forms the reflector of column k itself
  // (the same data and arithmetic in each, so no barrier for it), p = b A22 v with four
  // threads per row, then the rank-2 update; two barriers per step
  for (int k = 0; k + 2 < n; ++k) {
    const int L = n - k - 1;
    const float x0 = A[k + 1][k];
    float s = 0.f;
    for (int i = 1 + lane; i < L; i += 32) s = fmaf(A[k + 1 + i][k], A[k + 1 + i][k], s);
    s = warp_sum(s);
    float b = 0.f, alpha = x0;
    if (s != 0.f) {
      const float r = sqrtf(fmaf(x0, x0, s));
      alpha = x0 >= 0.f ? -r : r;
      b = 1.f / (alpha * (alpha - x0));
    }
    const float v0 = x0 - alpha;  // v = x - alpha e_1 (stored in A[k+1:, k] below)
    if (tid == 0) {
      sh.td[k] = A[k][k];
      sh.tbeta[k] = b;
      sh.te[k] = alpha;
    }
    if (b == 0.f) continue;  // every thread takes the same branch
    {  // p = b A22 v: row tid / 4, the quad's four partial sums added by shuffles
      const int ir = tid >> 2, q = tid & 3;
      float acc = 0.f;
      if (ir < L) {
        const int i = k + 1 + ir;
        for (int j = q; j < L; j += 4)
          acc = fmaf(A[i][k + 1 + j], j == 0 ? v0 : A[k + 1 + j][k], acc);
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (ir < L && q == 0) sh.tp[ir] = b * acc;
    }
    __syncthreads();
    float kk = 0.f;  // K = b p.v / 2, w = p - K v; A22 -= v w^T + w v^T
    for (int j = lane; j < L; j += 32) kk = fmaf(sh.tp[j], j == 0 ? v0 : A[k + 1 + j][k], kk);
    kk = 0.5f * b * warp_sum(kk);
    for (int i = warp; i < L; i += JT / 32) {
      const float vi = i == 0 ? v0 : A[k + 1 + i][k], wi = fmaf(-kk, vi, sh.tp[i]);
      for (int j = lane; j < L; j += 32) {
        const float vj = j == 0 ? v0 : A[k + 1 + j][k], wj = fmaf(-kk, vj, sh.tp[j]);
        A[k + 1 + i][k + 1 + j] -= fmaf(vi, wj, wi * vj);
      }
    }
    if (tid == 0) A[k + 1][k] = v0;  // every read of x0 happened before the barrier above
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      sh.td[n - 2] = A[n - 2][n - 2];
      sh.te[n - 2] = A[n - 1][n - 2];
    }
    sh.td[n - 1] = A[n - 1][n - 1];
    float lo = sh.td[0], hi = sh.td[0];
    for (int i = 0; i < n; ++i) {
      const float r = (i > 0 ? fabsf(sh.te[i - 1]) : 0.f) + (i + 1 < n ? fabsf(sh.te[i]) : 0.f);
      lo = fminf(lo, sh.td[i] - r);
      hi = fmaxf(hi, sh.td[i] + r);
      if (i + 1 < n) sh.te2[i] = sh.te[i] * sh.te[i];
    }
    sh.tlo = lo;
    sh.thi = hi;
  }
  __syncthreads();
  if (warp == 0) {  // segment starts: index 0 and i + 1 wherever e_i is negligible
    bool f0 = lane == 0, f1 = false;
    if (lane >= 1 && lane < n) {
      const int i = lane - 1;
      f0 = fabsf(sh.te[i]) <= 5.9604645e-8f * (fabsf(sh.td[i]) + fabsf(sh.td[i + 1]));
    }
    if (lane + 32 < n) {
      const int i = lane + 31;
      f1 = fabsf(sh.te[i]) <= 5.9604645e-8f * (fabsf(sh.td[i]) + fabsf(sh.td[i + 1]));
    }
    const unsigned m0 = __ballot_sync(0xffffffffu, f0), m1 = __ballot_sync(0xffffffffu, f1);
    if (f0 && lane >= 1) {
      sh.te[lane - 1] = 0.f;
      sh.te2[lane - 1] = 0.f;
    }
    if (f1) {
      sh.te[lane + 31] = 0.f;
      sh.te2[lane + 31] = 0.f;
    }
    if (lane == 0) sh.tsmask = (unsigned long long)m0 | ((unsigned long long)m1 << 32);
  }
  __syncthreads();
  const unsigned long long SEG = sh.tsmask;
  // segment [s, t) of index j
  auto seg_of = [&](int j, int &s0, int &t0) {
    const unsigned long long le = (j == 63) ? ~0ull : ((2ull << j) - 1ull);
    s0 = 63 - __clzll(SEG & le);
    const unsigned long long above = SEG & ~le;
    t0 = above ? __ffsll((long long)above) - 1 : n;
  };
  const float tnorm = fmaxf(fabsf(sh.tlo), fabsf(sh.thi));
  if (!(tnorm > 0.f)) {  // T = 0 (or not finite): any orthonormal basis
    for (int e = tid; e < n * 64; e += JT) {
      const int i = e >> 6, j = e & 63;
      if (j < n) sh.v[i][j] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    return;
  }
  // 2. eigenvalues: G threads per eigenvalue (a power of two dividing 32)
  {
    int G = 32;
    while (G > 1 && G * n > JT) G >>= 1;
    const int j = tid / G, g = tid - j * G;
    int s0 = 0, t0 = n;
    if (j < n) seg_of(j, s0, t0);
    const int jl = j - s0;
    const float pivmin = 1e-30f * fmaxf(1.f, tnorm * tnorm);
    float lo = sh.tlo - (2e-7f * tnorm + pivmin);
    float hi = sh.thi + (2e-7f * tnorm + pivmin);
    // each step shrinks the interval G + 1 times; enough steps for 2^-26 of it
    const int iters = G >= 16 ? 8 : (G >= 8 ? 9 : (G >= 4 ? 12 : (G >= 2 ? 17 : 26)));
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    for (int it = 0; it < iters; ++it) {
      const float x = lo + (hi - lo) * (float)(g + 1) / (float)(G + 1);
      int c = 0;
      if (j < n) {
        float q = sh.td[s0] - x;
        if (fabsf(q) < pivmin) q = -pivmin;
        c = q < 0.f;
        for (int i = s0 + 1; i < t0; ++i) {
          q = sh.td[i] - x - __fdividef(sh.te2[i - 1], q);
          if (fabsf(q) < pivmin) q = -pivmin;
          c += q < 0.f;
        }
      }
      // points with count <= jl lie below the segment's eigenvalue jl; counts grow with x
      const unsigned below = __ballot_sync(0xffffffffu, j < n && c <= jl) & gmask;
      const int t = __popc(below);
      const float nlo = t > 0 ? lo + (hi - lo) * (float)t / (float)(G + 1) : lo;
      const float nhi = t < G ? lo + (hi - lo) * (float)(t + 1) / (float)(G + 1) : hi;
      lo = nlo;
      hi = nhi;
    }
    if (j < n && g == 0) sh.tlam[j] = 0.5f * (lo + hi);
  }
  __syncthreads();
  if (warp == 0) {  // clusters: runs of eigenvalues of one segment with gaps <= 1e-4 ||T||
    const bool b0 = lane < n && (lane == 0 || ((SEG >> lane) & 1ull) ||
                                 sh.tlam[lane] - sh.tlam[lane - 1] > 1e-4f * tnorm);
    const bool b1 = lane + 32 < n && (((SEG >> (lane + 32)) & 1ull) ||
                                      sh.tlam[lane + 32] - sh.tlam[lane + 31] > 1e-4f * tnorm);
    const unsigned m0 = __ballot_sync(0xffffffffu, b0), m1 = __ballot_sync(0xffffffffu, b1);
    if (lane == 0) sh.tcmask = (unsigned long long)m0 | ((unsigned long long)m1 << 32);
  }
  __syncthreads();
  // 3. inverse iteration (z in column j of v, the LDL^T multipliers in column j of a[1])
  float(*Lm)[JMAX + 1] = sh.a[1];
  const float pmin = 1.1920929e-7f * tnorm;
  int s0 = 0, t0 = n;
  if (tid < n) {
    const int j = tid;
    seg_of(j, s0, t0);
    for (int i = 0; i < n; ++i) {  // a start vector of pseudo-random entries in [-1, 1]
      unsigned h = (unsigned)(i + 1) * 2654435761u ^ (unsigned)(j + 1) * 40503u;
      h ^= h >> 15;
      h *= 2246822519u;
      h ^= h >> 13;
      sh.v[i][j] = (i >= s0 && i < t0) ? (float)(h & 0xffffff) * (2.f / 16777216.f) - 1.f : 0.f;
    }
  }
  for (int step = 0; step < 2; ++step) {
    if (tid < n) {
      const int j = tid;
      const float lam = sh.tlam[j];
      float dt = sh.td[s0] - lam;
      if (fabsf(dt) < pmin) dt = dt < 0.f ? -pmin : pmin;
      float y = sh.v[s0][j];
      for (int i = s0; i + 1 < t0; ++i) {
        const float l = __fdividef(sh.te[i], dt);
        Lm[i][j] = l;
        const float yn = fmaf(-l, y, sh.v[i + 1][j]);
        sh.v[i][j] = __fdividef(y, dt);
        float dn = fmaf(-l, sh.te[i], sh.td[i + 1] - lam);
        if (fabsf(dn) < pmin) dn = dn < 0.f ? -pmin : pmin;
        dt = dn;
        y = yn;
      }
      float z = __fdividef(y, dt);
      sh.v[t0 - 1][j] = z;
      float nrm = z * z;
      for (int i = t0 - 2; i >= s0; --i) {
        z = fmaf(-Lm[i][j], z, sh.v[i][j]);
        sh.v[i][j] = z;
        nrm = fmaf(z, z, nrm);
      }
      const float sc = rsqrtf(nrm);
      for (int i = s0; i < t0; ++i) sh.v[i][j] *= sc;
    }
    __syncthreads();
    // modified Gram-Schmidt inside each cluster, one warp per cluster
    {
      const unsigned long long B = sh.tcmask;
      const int ncl = __popcll(B);
      for (int c = warp; c < ncl; c += JT / 32) {
        unsigned long long bb = B;  // the c-th set bit of B starts cluster c
        for (int q = 0; q < c; ++q) bb &= bb - 1;
        const int f0 = __ffsll((long long)bb) - 1;
        const unsigned long long rest = (f0 == 63) ? 0ull : (B & ~((2ull << f0) - 1ull));
        const int f1 = rest ? __ffsll((long long)rest) - 1 : n;
        for (int jj = f0 + 1; jj < f1; ++jj) {
          for (int kq = f0; kq < jj; ++kq) {
            float s = 0.f;
            for (int i = lane; i < n; i += 32) s = fmaf(sh.v[i][kq], sh.v[i][jj], s);
            s = warp_sum(s);
            for (int i = lane; i < n; i += 32) sh.v[i][jj] = fmaf(-s, sh.v[i][kq], sh.v[i][jj]);
          }
          float s = 0.f;
          for (int i = lane; i < n; i += 32) s = fmaf(sh.v[i][jj], sh.v[i][jj], s);
          const float sc = rsqrtf(warp_sum(s));
          for (int i = lane; i < n; i += 32) sh.v[i][jj] *= sc;
        }
      }
    }
    __syncthreads();
  }
  // 4. X = H_0 (H_1 (... H_{n-3} Z)) for columns c0 .. c1 - 1: P threads per column (P a
  // power of two, P (c1 - c0) <= JT)
  {
    const int nc = c1 - c0;
    int P = 32;
    while (P > 1 && P * nc > JT) P >>= 1;
    const int j = c0 + tid / P, part = tid - (tid / P) * P;
    for (int k = n - 3; k >= 0; --k) {
      const float b = sh.tbeta[k];
      if (b == 0.f) continue;
      float u = 0.f;
      if (j < c1)
        for (int i = k + 1 + part; i < n; i += P) u = fmaf(A[i][k], sh.v[i][j], u);
      for (int o = 1; o < P; o <<= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
      if (j < c1)
        for (int i = k + 1 + part; i < n; i += P) sh.v[i][j] = fmaf(-b * u, A[i][k], sh.v[i][j]);
    }
  }
  __syncthreads();
}

// gather a square m x m array from column owners: dst[i][j] = owner(j)'s src[i][loc(j)]
#define GATHER_COLS(dst, src)                                                         \
  for (int i = warp; i < m; i += JT / 32) {                                           \
    for (int j = lane; j < m; j += 32) {                                              \
      const int o = sh.owner[j];                                                      \
      dst[i][j] = (o == rank) ? src[i][sh.loc[j]] : *peer(&src[i][sh.loc[j]], o);     \
    }                                                                                 \
  }

__global__ void __cluster_dims__(JCL, 1, 1) __launch_bounds__(JT)
k_rr_mixed(const double *__restrict__ G, int m, int ldg, double *theta, double *Yout, int ldy,
           int mp, int *__restrict__ stat, double tol_abs, double *Arot, int refine_max) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MixedSmem &sh = *reinterpret_cast<MixedSmem *>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int R = (m + JCL - 1) / JCL;  // rows (columns) per CTA
  const int r0 = rank * R;
  const int nown = max(0, min(R, m - r0));
  const int nn = (m + 1) & ~1;
  auto peer = [&](const auto *p, int r) { return cluster.map_shared_rank(p, (unsigned)r); };

  // ---- A0: own rows, ||A0||_F, then the other rows from their owners
  if (tid < JMAX) {
    sh.owner[tid] = tid / R;
    sh.loc[tid] = tid - (tid / R) * R;
  }
  double f = 0.0;
  for (int e = tid; e < nown * m; e += JT) {
    const int il = e / m, j = e - il * m;
    const double v = a0_entry(G, ldg, theta, Yout, ldy, mp, Arot, r0 + il, j);
    sh.A0[r0 + il][j] = v;
    f = fma(v, v, f);
  }
  for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
  if (lane == 0) sh.dred[warp] = f;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < JT / 32; ++w) t += sh.dred[w];
    sh.norm2 = t;
  }
  cluster.sync();
  for (int i = warp; i < m; i += JT / 32) {
    const int o = sh.owner[i];
    if (o == rank) continue;
    for (int j = lane; j < m; j += 32) sh.A0[i][j] = *peer(&sh.A0[i][j], o);
  }
  if (tid == 0) {
    double t = 0.0;
    for (int c = 0; c < JCL; ++c) t += *peer(&sh.norm2, c);
    const double nrm = sqrt(t);
    sh.nrmA = nrm;
    sh.inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    sh.thr_bits = abs_bits(fmax(8.9e-16 * nrm, tol_abs));
    sh.solves32 = 0;
    sh.groups_rot = 0;
  }
  __syncthreads();
  const double normA = sh.nrmA;
  const unsigned long long thr_bits = sh.thr_bits;
  // 4 m u: the rounding floor of I - X^T X for an orthonormal X
  const unsigned long long orth_bits = abs_bits(4.0 * m * 1.1102230246251565e-16);

  // ---- FP32 eigenvectors of A0 / ||A0||_F (replicated)
  {
    const double inv = sh.inv;
    for (int e = tid; e < nn * 64; e += JT) {
      const int i = e >> 6, j = e & 63;
      if (j >= nn) continue;
      sh.a[0][i][j] = (i < m && j < m) ? (float)(sh.A0[i][j] * inv) : 0.f;
      sh.v[i][j] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();
    // every CTA finds the same eigenvalues and segment vectors; each back-transforms its
    // own columns (CTA r: r R .. r R + R - 1) and reads the others' from their owners
    eig32(sh, m, min(r0, m), min(r0 + R, m));
    if (tid == 0) sh.solves32 += 1;
    cluster.sync();
    for (int e = tid; e < m * 64; e += JT) {
      const int i = e >> 6, j = e & 63;
      if (j >= m) continue;
      const int o = sh.owner[j];
      sh.X[i][j] = (double)((o == rank) ? sh.v[i][j] : *peer(&sh.v[i][j], o));
    }
    // no CTA overwrites its v until every peer has read it (the group rotations reuse it)
    cluster.sync();
  }

  // ---- FP64 refinement; CTA r owns columns r0 .. r0 + nown - 1 of W, S, R, E and X
  bool converged = false;
  int it = 0;
  for (; it <= refine_max; ++it) {
    // (1) own columns of W = A0 X, then of S = X^T W and R = I - X^T X (R is exactly
    // symmetric: r_ij and r_ji are the same products summed in the same order)
    for (int e = tid; e < nown * m; e += JT) {
      const int jl = e / m, k = e - jl * m, gj = r0 + jl;
      double s0 = 0.0, s1 = 0.0;
      int i = 0;
      for (; i + 1 < m; i += 2) {
        s0 = fma(sh.A0[k][i], sh.X[i][gj], s0);
        s1 = fma(sh.A0[k][i + 1], sh.X[i + 1][gj], s1);
      }
      if (i < m) s0 = fma(sh.A0[k][i], sh.X[i][gj], s0);
      sh.W[k][jl] = s0 + s1;
    }
    __syncthreads();
    unsigned long long rb = 0;
    for (int e = tid; e < nown * m; e += JT) {
      const int jl = e / m, i = e - jl * m, gj = r0 + jl;
      double s0 = 0.0, s1 = 0.0, t0 = 0.0, t1 = 0.0;
      int k = 0;
      for (; k + 1 < m; k += 2) {
        s0 = fma(sh.X[k][i], sh.W[k][jl], s0);
        t0 = fma(sh.X[k][i], sh.X[k][gj], t0);
        s1 = fma(sh.X[k + 1][i], sh.W[k + 1][jl], s1);
        t1 = fma(sh.X[k + 1][i], sh.X[k + 1][gj], t1);
      }
      if (k < m) {
        s0 = fma(sh.X[k][i], sh.W[k][jl], s0);
        t0 = fma(sh.X[k][i], sh.X[k][gj], t0);
      }
      sh.S[i][jl] = s0 + s1;
      const double r = ((i == gj) ? 1.0 : 0.0) - (t0 + t1);
      sh.R[i][jl] = r;
      const unsigned long long b = abs_bits(r);
      rb = b > rb ? b : rb;
    }
    rb = cta_max_u64(rb, sh.bred);
    if (tid == 0) sh.rmax = rb;
    cluster.sync();
    // (2) S gathered and symmetrised, r_ii, max |r| over the cluster
    GATHER_COLS(sh.F, sh.S)
    if (tid < m) {
      const int o = sh.owner[tid];
      sh.rd[tid] = (o == rank) ? sh.R[tid][sh.loc[tid]] : *peer(&sh.R[tid][sh.loc[tid]], o);
    }
    if (tid == 0) {
      unsigned long long t = 0;
      for (int c = 0; c < JCL; ++c) {
        const unsigned long long u = *peer(&sh.rmax, c);
        t = u > t ? u : t;
      }
      sh.rall_bits = t;
    }
    __syncthreads();
    unsigned long long ob = 0;
    for (int e = tid; e < m * 64; e += JT) {
      const int i = e >> 6, j = e & 63;
      if (j <= i || j >= m) continue;
      const double s = 0.5 * (sh.F[i][j] + sh.F[j][i]);
      sh.F[i][j] = s;
      sh.F[j][i] = s;
      const unsigned long long b = abs_bits(s);
      ob = b > ob ? b : ob;
    }
    ob = cta_max_u64(ob, sh.bred);  // (its barriers also complete the symmetrisation)
    if (ob <= thr_bits && sh.rall_bits <= orth_bits) {
      converged = true;
      break;
    }
    if (it == refine_max) break;
    // (3) lambda, delta, ascending order, groups (runs of sorted lambda with gaps <= delta)
    if (tid < m) {
      const double l = sh.F[tid][tid] / (1.0 - sh.rd[tid]);
      sh.lam[tid] = l;
      sh.key[tid] = order_key(l);
    }
    if (tid == 0)
      sh.delta = 2.0 * m * (__longlong_as_double((long long)ob) +
                            normA * __longlong_as_double((long long)sh.rall_bits));
    __syncthreads();
    if (tid < m) {
      const long long ki = sh.key[tid];
      int rk = 0;
      for (int j = 0; j < m; ++j) rk += (sh.key[j] < ki) || (sh.key[j] == ki && j < tid);
      sh.order[rk] = tid;
      sh.ipos[tid] = rk;
    }
    __syncthreads();
    if (warp == 0) {
      const int t0 = lane, t1 = lane + 32;
      const bool b0 = t0 < m && (t0 == 0 || sh.lam[sh.order[t0]] - sh.lam[sh.order[t0 - 1]] > sh.delta);
      const bool b1 = t1 < m && (sh.lam[sh.order[t1]] - sh.lam[sh.order[t1 - 1]] > sh.delta);
      const unsigned m0 = __ballot_sync(0xffffffffu, b0), m1 = __ballot_sync(0xffffffffu, b1);
      if (lane == 0) sh.gmask = (unsigned long long)m0 | ((unsigned long long)m1 << 32);
    }
    __syncthreads();
    if (tid < m) {  // group starts are the set bits of gmask
      const unsigned long long B = sh.gmask;
      const unsigned long long le = (tid == 63) ? ~0ull : ((2ull << tid) - 1);
      const int first = 63 - __clzll(B & le);
      const unsigned long long above = B & ~le;
      const int next = above ? __ffsll((long long)above) - 1 : m;
      sh.gfirst[tid] = first;
      sh.gsize[tid] = next - first;
      sh.flag[tid] = (next - first) >= 2;
    }
    __syncthreads();
    // (4) own columns of E, and the group blocks T_ij = s_ij + (lambda_i + lambda_j) r_ij / 2
    // (T_ii = lambda_i): the block predicted for after the update, built here because it
    // reads the other CTAs' R, which they overwrite after the next cluster barrier
    for (int e = tid; e < nown * m; e += JT) {
      const int jl = e / m, i = e - jl * m, gj = r0 + jl;
      const double r = sh.R[i][jl];  // r_{i, gj}
      double ev;
      if (sh.gfirst[sh.ipos[i]] == sh.gfirst[sh.ipos[gj]])
        ev = 0.5 * r;
      else
        ev = (sh.F[i][gj] + sh.lam[gj] * r) / (sh.lam[gj] - sh.lam[i]);
      sh.E[i][jl] = ev;
    }
    warp0_prefix(sh.flag, m, sh.cnt);
    __syncthreads();
    if (tid < m && sh.flag[tid]) sh.ml[sh.cnt[tid] - 1] = tid;
    if (tid == 0) sh.nm = (m > 0) ? sh.cnt[m - 1] : 0;
    __syncthreads();
    const int nm = sh.nm;
    if (tid < nm) {
      const int u = sh.ml[tid];
      const int b = tid - (u - sh.gfirst[u]);
      sh.mbeg[tid] = b;
      sh.mend[tid] = b + sh.gsize[u];
      sh.cscale[tid] = 0u;
      sh.coff[tid] = 0ull;
    }
    __syncthreads();
    for (int e = tid; e < nm * 64; e += JT) {
      const int x = e >> 6, z = e & 63;
      if (z < sh.mbeg[x] || z >= sh.mend[x]) continue;
      const int i = sh.order[sh.ml[x]], j = sh.order[sh.ml[z]];
      double t, d;
      if (x == z) {
        t = sh.lam[i];
        d = t - sh.lam[sh.order[sh.ml[sh.mbeg[x]]]];
      } else {
        const int o = sh.owner[j];
        const double r = (o == rank) ? sh.R[i][sh.loc[j]] : *peer(&sh.R[i][sh.loc[j]], o);
        t = fma(0.5 * (sh.lam[i] + sh.lam[j]), r, sh.F[i][j]);
        d = t;
        atomicMax(&sh.coff[sh.mbeg[x]], abs_bits(t));
      }
      sh.P[x][z] = t;
      atomicMax(&sh.cscale[sh.mbeg[x]], __float_as_uint(fabsf((float)d)));
    }
    // (5) own columns of X (I + E)
    for (int e = tid; e < nown * m; e += JT) {
      const int jl = e / m, k = e - jl * m, gj = r0 + jl;
      double s0 = sh.X[k][gj], s1 = 0.0;
      int i = 0;
      for (; i + 1 < m; i += 2) {
        s0 = fma(sh.X[k][i], sh.E[i][jl], s0);
        s1 = fma(sh.X[k][i + 1], sh.E[i + 1][jl], s1);
      }
      if (i < m) s0 = fma(sh.X[k][i], sh.E[i][jl], s0);
      sh.Xn[k][jl] = s0 + s1;
    }
    cluster.sync();
    // (6) X gathered from the owners of its columns
    GATHER_COLS(sh.X, sh.Xn)
    // (7) groups whose predicted block has an off-diagonal above thr: the FP32 eigensolver
    // on the block shifted by its first eigenvalue estimate and scaled to unit max entry
    if (tid < nm)
      sh.flag[tid] = (sh.coff[sh.mbeg[tid]] > thr_bits) && (sh.cscale[sh.mbeg[tid]] != 0u);
    __syncthreads();
    warp0_prefix(sh.flag, nm, sh.cnt);
    __syncthreads();
    if (tid < nm && sh.flag[tid]) sh.clist[sh.cnt[tid] - 1] = tid;
    if (tid == 0) sh.nc = (nm > 0) ? sh.cnt[nm - 1] : 0;
    __syncthreads();
    const int nc = sh.nc;
    if (nc == 0) continue;
    if (tid < nc) {  // a rotated group is contiguous in clist as it is in ml
      const int x = sh.clist[tid];
      const int b = tid - (x - sh.mbeg[x]);
      sh.cbeg[tid] = b;
      sh.cend[tid] = b + (sh.mend[x] - sh.mbeg[x]);
      if (x == sh.mbeg[x]) atomicAdd(&sh.groups_rot, 1);
    }
    __syncthreads();
    const int ncc = (nc + 1) & ~1;
    for (int e = tid; e < ncc * 64; e += JT) {
      const int y = e >> 6, w = e & 63;
      if (w >= ncc) continue;
      float a = 0.f;
      if (y < nc && w >= sh.cbeg[y] && w < sh.cend[y]) {
        const int x = sh.clist[y], z = sh.clist[w], g0 = sh.mbeg[x];
        const double d = (y == w) ? sh.P[x][z] - sh.lam[sh.order[sh.ml[g0]]] : sh.P[x][z];
        a = (float)d / __uint_as_float(sh.cscale[g0]);
      }
      sh.a[0][y][w] = a;
      sh.v[y][w] = (y == w) ? 1.f : 0.f;
    }
    __syncthreads();
    eig32(sh, nc);
    if (tid == 0) sh.solves32 += 1;
    // W_J in FP64 (into P, clist-indexed), two Newton-Schulz steps W <- W (3 I - W^T W) / 2
    for (int e = tid; e < nc * 64; e += JT) {
      const int y = e >> 6, w = e & 63;
      if (w < nc) sh.P[y][w] = (w >= sh.cbeg[y] && w < sh.cend[y]) ? (double)sh.v[y][w] : 0.0;
    }
    __syncthreads();
    {
      // Z = W M in the FP32 Jacobi's buffers (free now; the same size as a double array)
      double(*Z)[LD] = reinterpret_cast<double(*)[LD]>(&sh.a[0][0][0]);
      for (int step = 0; step < 2; ++step) {
        for (int e = tid; e < nc * 64; e += JT) {  // F = M = W^T W on the blocks
          const int y = e >> 6, w = e & 63;
          if (w < sh.cbeg[y] || w >= sh.cend[y]) continue;
          double s = 0.0;
          for (int z = sh.cbeg[y]; z < sh.cend[y]; ++z) s = fma(sh.P[z][y], sh.P[z][w], s);
          sh.F[y][w] = s;
        }
        __syncthreads();
        for (int e = tid; e < nc * 64; e += JT) {  // Z = W M
          const int y = e >> 6, w = e & 63;
          if (w < sh.cbeg[y] || w >= sh.cend[y]) continue;
          double s = 0.0;
          for (int z = sh.cbeg[y]; z < sh.cend[y]; ++z) s = fma(sh.P[y][z], sh.F[z][w], s);
          Z[y][w] = s;
        }
        __syncthreads();
        for (int e = tid; e < nc * 64; e += JT) {  // W = 1.5 W - 0.5 Z
          const int y = e >> 6, w = e & 63;
          if (w >= sh.cbeg[y] && w < sh.cend[y]) sh.P[y][w] = fma(-0.5, Z[y][w], 1.5 * sh.P[y][w]);
        }
        __syncthreads();
      }
    }
    // X_J <- X_J W_J: new columns into F, then back into X
    for (int e = tid; e < m * 64; e += JT) {
      const int k = e >> 6, y = e & 63;
      if (y >= nc) continue;
      double s = 0.0;
      for (int z = sh.cbeg[y]; z < sh.cend[y]; ++z)
        s = fma(sh.X[k][sh.order[sh.ml[sh.clist[z]]]], sh.P[z][y], s);
      sh.F[k][y] = s;
    }
    __syncthreads();
    for (int e = tid; e < m * 64; e += JT) {
      const int k = e >> 6, y = e & 63;
      if (y < nc) sh.X[k][sh.order[sh.ml[sh.clist[y]]]] = sh.F[k][y];
    }
    __syncthreads();
  }

  if (!converged) {
    // inputs untouched: solve by FP64 Jacobi in the same shared memory once every CTA is
    // done reading this one's buffers
    if (stat && rank == 0 && tid == 0) {
      atomicAdd(&stat[3], 1);
      atomicAdd(&stat[4], sh.solves32);
      atomicAdd(&stat[5], it);
      atomicAdd(&stat[6], sh.groups_rot);
      atomicAdd(&stat[7], 1);
    }
    cluster.sync();
    jacobi64(*reinterpret_cast<JacobiSmem *>(smem_raw), cluster, G, m, ldg, theta, Yout, ldy, mp,
             stat, tol_abs, Arot);
    return;
  }

  // ---- outputs: ascending theta = diag(S); Y = Q0 X[:, order]; Arot = S in that order
  if (tid < m) sh.key[tid] = order_key(sh.F[tid][tid]);
  __syncthreads();
  if (tid < m) {
    const long long ki = sh.key[tid];
    int rk = 0;
    for (int j = 0; j < m; ++j) rk += (sh.key[j] < ki) || (sh.key[j] == ki && j < tid);
    sh.order[rk] = tid;
    sh.ipos[tid] = rk;
  }
  __syncthreads();
  double yv[JOUT];
#pragma unroll
  for (int q = 0; q < JOUT; ++q) {
    const int e = tid + q * JT;
    double v = 0.0;
    if (e < nown * m) {
      const int il = e / m, j = e - il * m, gi = r0 + il;
      const int pj = sh.order[j];
      if (gi < mp) {
#pragma unroll 8
        for (int a = 0; a < mp; ++a) v = fma(Yout[(long long)a * ldy + gi], sh.X[a][pj], v);
      } else {
        v = sh.X[gi][pj];
      }
    }
    yv[q] = v;
  }
  cluster.sync();  // every CTA is done reading the previous Y
#pragma unroll
  for (int q = 0; q < JOUT; ++q) {
    const int e = tid + q * JT;
    if (e < nown * m) {
      const int il = e / m, j = e - il * m;
      Yout[(long long)j * ldy + r0 + il] = yv[q];
    }
  }
  if (Arot)
    for (int e = tid; e < nown * m; e += JT) {
      const int il = e / m, c = e - il * m, gi = r0 + il;
      Arot[(long long)sh.ipos[c] * ldy + sh.ipos[gi]] = sh.F[gi][c];
    }
  if (rank == 0) {
    for (int j = tid; j < m; j += JT) theta[j] = sh.F[sh.order[j]][sh.order[j]];
    if (stat && tid == 0) {
      atomicAdd(&stat[3], 1);
      atomicAdd(&stat[4], sh.solves32);
      atomicAdd(&stat[5], it);
      atomicAdd(&stat[6], sh.groups_rot);
    }
  }
}
#undef GATHER_COLS

}  // namespace

void launch_jacobi_eigh(const double *G, int m, int ldg, double *theta, double *Y, int ldy,
                        cudaStream_t s, int mp, int *stat, double tol_abs, double *Arot) {
  count_launch();
  launch_pdl(k_jacobi, JCL, JT, 0, s, G, m, ldg, theta, Y, ldy,
             mp < m ? mp : 0, stat, tol_abs, Arot);
}

void launch_rr_eigh(const double *G, int m, int ldg, double *theta, double *Y, int ldy,
                    cudaStream_t s, int mp, int *stat, double tol_abs, double *Arot, int method,
                    int refine_max) {
  if (method == TPS_RR_JACOBI64) {
    launch_jacobi_eigh(G, m, ldg, theta, Y, ldy, s, mp, stat, tol_abs, Arot);
    return;
  }
  static std::atomic<unsigned> attr_done{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned bit = 1u << (dev & 31);
  if (!(attr_done.load() & bit)) {
    cudaFuncSetAttribute(k_rr_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(MixedSmem));
    attr_done.fetch_or(bit);
  }
  count_launch();
  launch_pdl(k_rr_mixed, JCL, JT, sizeof(MixedSmem), s, G, m, ldg, theta, Y, ldy,
             mp < m ? mp : 0, stat,
                                                 tol_abs, Arot, refine_max > 0 ? refine_max : kRefineMax);
}

}  // namespace tps
