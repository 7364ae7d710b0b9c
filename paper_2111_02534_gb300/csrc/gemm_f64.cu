// FP64 mode-product GEMMs for the H-apply (Eq. tensor_op1D, Eq. tensor_op2D) and the
// fast-diagonalisation preconditioner (Sec. 4.2), with the pointwise terms fused into
// the epilogue.
//
// One kernel template computes, for every batch z,
//     C[z] (M x Nc) = sum over phases p of A_p[z] (M x K_p) * B_p[z] (K_p x Nc)
// followed by an epilogue: plain store, + (V - theta) * psi (H-apply), division by a
// Kronecker sum of eigenvalues (preconditioner), or accumulation into C.  Every
// operand is row-major with unit column stride, a row stride and a batch stride (0 =
// shared by all batches), so a mode-k product of a C-ordered tensor is a batched GEMM
// without any transpose (the two extra passes of Sec. 3.3 disappear).
//
// Two phases share one accumulator: in 1D the x product K_x * P and the y product
// P * K_y^T of the same output tile are summed in registers before the V term is
// added, so each H-apply is one kernel launch that reads psi once per tile.
//
// GB300 has no FP64 tensor-core path (tcgen05 has no f64 kind), so these kernels
// run on the FP64 FMA pipe: each thread owns a 4x4 register tile, operands are
// staged through double-buffered shared memory with the next k-slab prefetched into
// registers while the current one is consumed.
#include <cstring>

#include "tps_internal.h"

namespace tps {
namespace {

struct Opnd {
  const double *p;
  long long rs;  // row stride
  long long bs;  // batch stride (0: shared)
};

enum Epi { EPI_STORE = 0, EPI_HAPPLY = 1, EPI_DIVIDE2 = 2, EPI_ACCUM = 3, EPI_DIVIDE4 = 4 };

struct GemmArgs {
  int M, Nc, batch, nphase;
  int K[2];
  Opnd A[2], B[2];
  double *C;
  long long ldc, bsc;
  int epi;
  // EPI_HAPPLY: C += (V[(z % vmod) * vbs + m * ldv + n] - theta_z) * E[z][m][n]
  Opnd E;
  const double *V;
  long long ldv, vbs, vmod;
  const double *theta;
  long long theta_div;
  double theta0;
  // EPI_DIVIDE2: C /= (lamM[m] + lamN[n] - sigma)
  // EPI_DIVIDE4: C /= (lamM[m] + l1[n / (n2*n3)] + l2[(n / n3) % n2] + l3[n % n3] - sigma)
  const double *lamM, *lamN, *lam2, *lam3;
  int n2, n3;
  double sigma;
  int tiles_m, tiles_n;
};

constexpr int TK = 16;

template <int TM, int TN>
__global__ void __launch_bounds__((TM / 4) * (TN / 4))
k_gemm_f64(const GemmArgs g) {
  constexpr int NT = (TM / 4) * (TN / 4);
  constexpr int LA = (TM * TK + NT - 1) / NT;  // A elements staged per thread
  constexpr int LB = (TK * TN + NT - 1) / NT;  // B elements staged per thread
  __shared__ double As[2][TK][TM + 1];
  __shared__ double Bs[2][TK][TN];

  const int tid = threadIdx.x;
  const int tn = tid % (TN / 4);
  const int tm = tid / (TN / 4);
  long long bid = blockIdx.x;
  const int tiles = g.tiles_m * g.tiles_n;
  const long long z = bid / tiles;
  const int t = (int)(bid % tiles);
  const int m0 = (t / g.tiles_n) * TM;
  const int n0 = (t % g.tiles_n) * TN;

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  const int ks0 = (g.K[0] + TK - 1) / TK;
  const int nstage = ks0 + (g.nphase > 1 ? (g.K[1] + TK - 1) / TK : 0);

  double ra[LA], rb[LB];
  auto fetch = [&](int stage) {
    const int ph = stage < ks0 ? 0 : 1;
    const int k0 = (ph == 0 ? stage : stage - ks0) * TK;
    const int Kp = g.K[ph];
    const double *Ap = g.A[ph].p + z * g.A[ph].bs;
    const double *Bp = g.B[ph].p + z * g.B[ph].bs;
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int e = tid + l * NT;
      const int m = e / TK, k = e % TK;
      double v = 0.0;
      if (e < TM * TK && m0 + m < g.M && k0 + k < Kp) v = Ap[(long long)(m0 + m) * g.A[ph].rs + k0 + k];
      ra[l] = v;
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int e = tid + l * NT;
      const int k = e / TN, n = e % TN;
      double v = 0.0;
      if (e < TK * TN && k0 + k < Kp && n0 + n < g.Nc) v = Bp[(long long)(k0 + k) * g.B[ph].rs + n0 + n];
      rb[l] = v;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int e = tid + l * NT;
      if (e < TM * TK) As[buf][e % TK][e / TK] = ra[l];
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int e = tid + l * NT;
      if (e < TK * TN) Bs[buf][e / TN][e % TN] = rb[l];
    }
  };

  if (nstage > 0) {
    fetch(0);
    stash(0);
  }
  __syncthreads();
  for (int s = 0; s < nstage; ++s) {
    const int buf = s & 1;
    if (s + 1 < nstage) fetch(s + 1);
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[buf][k][tm * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[buf][k][tn * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (s + 1 < nstage) stash(buf ^ 1);
    __syncthreads();
  }

  // epilogue
  double th = 0.0;
  if (g.epi == EPI_HAPPLY) th = g.theta ? g.theta[z / g.theta_div] : g.theta0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + tm * 4 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tn * 4 + j;
      if (n >= g.Nc) continue;
      double c = acc[i][j];
      double *dst = g.C + z * g.bsc + (long long)m * g.ldc + n;
      if (g.epi == EPI_HAPPLY) {
        const double v = g.V[(z % g.vmod) * g.vbs + (long long)m * g.ldv + n];
        const double p = g.E.p[z * g.E.bs + (long long)m * g.E.rs + n];
        c = fma(v - th, p, c);
      } else if (g.epi == EPI_DIVIDE2) {
        c = c / (g.lamM[m] + g.lamN[n] - g.sigma);
      } else if (g.epi == EPI_DIVIDE4) {
        const int n23 = g.n2 * g.n3;
        const double d = g.lamM[m] + g.lamN[n / n23] + g.lam2[(n / g.n3) % g.n2] + g.lam3[n % g.n3];
        c = c / (d - g.sigma);
      } else if (g.epi == EPI_ACCUM) {
        c += *dst;
      }
      *dst = c;
    }
  }
}

int pick_tile(int extent) {
  if (extent <= 32) return 32;
  if (extent % 64 == 0) return 64;
  if (extent % 48 == 0) return 48;
  if (extent <= 48) return 48;
  return 64;
}

template <int TM, int TN>
void run(GemmArgs g, cudaStream_t s) {
  g.tiles_m = (g.M + TM - 1) / TM;
  g.tiles_n = (g.Nc + TN - 1) / TN;
  const long long blocks = (long long)g.batch * g.tiles_m * g.tiles_n;
  if (blocks <= 0) return;
  count_launch();
  k_gemm_f64<TM, TN><<<(unsigned)blocks, (TM / 4) * (TN / 4), 0, s>>>(g);
}

void gemm(GemmArgs g, cudaStream_t s) {
  const int tm = pick_tile(g.M), tn = pick_tile(g.Nc);
#define TPS_TILE_CASE(A, B) \
  if (tm == A && tn == B) return run<A, B>(g, s);
  TPS_TILE_CASE(64, 64) TPS_TILE_CASE(64, 48) TPS_TILE_CASE(64, 32)
  TPS_TILE_CASE(48, 64) TPS_TILE_CASE(48, 48) TPS_TILE_CASE(48, 32)
  TPS_TILE_CASE(32, 64) TPS_TILE_CASE(32, 48) TPS_TILE_CASE(32, 32)
#undef TPS_TILE_CASE
}

GemmArgs base_args() {
  GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.vmod = 1;
  g.theta_div = 1;
  return g;
}

// One left mode product: C[z] = A (M x M, shared) * B[z] (M x Nc), B rows strided by rs.
GemmArgs left(const double *A, int M, const double *B, long long Nc, long long rs, long long bs,
              double *C, int batch) {
  GemmArgs g = base_args();
  g.M = M;
  g.Nc = (int)Nc;
  g.batch = batch;
  g.nphase = 1;
  g.K[0] = M;
  g.A[0] = {A, M, 0};
  g.B[0] = {B, rs, bs};
  g.C = C;
  g.ldc = rs;
  g.bsc = bs;
  return g;
}

// One right mode product over all rows: C (rows x n) = A (rows x n) * B (n x n).
GemmArgs right(const double *A, long long rows, int n, const double *B, double *C) {
  GemmArgs g = base_args();
  g.M = (int)rows;
  g.Nc = n;
  g.batch = 1;
  g.nphase = 1;
  g.K[0] = n;
  g.A[0] = {A, n, 0};
  g.B[0] = {B, n, 0};
  g.C = C;
  g.ldc = n;
  g.bsc = 0;
  return g;
}

// right product split into batches when the row count would overflow int
void right_batched(const double *A, long long rows, int n, const double *B, double *C,
                   cudaStream_t s) {
  const long long chunk = 1LL << 24;
  for (long long r0 = 0; r0 < rows; r0 += chunk) {
    const long long r = rows - r0 < chunk ? rows - r0 : chunk;
    gemm(right(A + r0 * n, r, n, B, C + r0 * n), s);
  }
}

}  // namespace

void launch_apply_h(const DevOperator &op, const double *psi, double *out, int nvec,
                    const double *theta_dev, double theta, cudaStream_t s) {
  if (nvec <= 0) return;
  if (op.nmodes == 2) {
    const int nx = op.n[0], ny = op.n[1];
    GemmArgs g = base_args();
    g.M = nx;
    g.Nc = ny;
    g.batch = nvec;
    g.nphase = 2;
    g.K[0] = nx;
    g.A[0] = {op.K[0], nx, 0};
    g.B[0] = {psi, ny, op.N};
    g.K[1] = ny;
    g.A[1] = {psi, ny, op.N};
    g.B[1] = {op.KT[1], ny, 0};
    g.C = out;
    g.ldc = ny;
    g.bsc = op.N;
    g.epi = EPI_HAPPLY;
    g.E = {psi, ny, op.N};
    g.V = op.V;
    g.ldv = ny;
    g.vbs = 0;
    g.vmod = 1;
    g.theta = theta_dev;
    g.theta_div = 1;
    g.theta0 = theta;
    gemm(g, s);
    return;
  }
  // 2D: [v][x1][x2][y1][y2]
  const int n0 = op.n[0], n1 = op.n[1], n2 = op.n[2], n3 = op.n[3];
  const long long s23 = (long long)n2 * n3, s123 = (long long)n1 * s23;
  {  // fused y1 + y2 products over every (v, x1, x2) slab, V and theta in the epilogue
    GemmArgs g = base_args();
    g.M = n2;
    g.Nc = n3;
    g.batch = nvec * n0 * n1;
    g.nphase = 2;
    g.K[0] = n2;
    g.A[0] = {op.K[2], n2, 0};
    g.B[0] = {psi, n3, s23};
    g.K[1] = n3;
    g.A[1] = {psi, n3, s23};
    g.B[1] = {op.KT[3], n3, 0};
    g.C = out;
    g.ldc = n3;
    g.bsc = s23;
    g.epi = EPI_HAPPLY;
    g.E = {psi, n3, s23};
    g.V = op.V;
    g.ldv = n3;
    g.vbs = s23;
    g.vmod = (long long)n0 * n1;
    g.theta = theta_dev;
    g.theta_div = (long long)n0 * n1;
    g.theta0 = theta;
    gemm(g, s);
  }
  {  // x2 product, accumulated
    GemmArgs g = left(op.K[1], n1, psi, s23, s23, s123, out, nvec * n0);
    g.epi = EPI_ACCUM;
    gemm(g, s);
  }
  {  // x1 product, accumulated
    GemmArgs g = left(op.K[0], n0, psi, s123, s123, op.N, out, nvec);
    g.epi = EPI_ACCUM;
    gemm(g, s);
  }
}

void launch_apply_prec(const DevOperator &op, const double *r, double *out, int nvec,
                       double sigma, ApplyWorkspace &ws, cudaStream_t s) {
  if (nvec <= 0) return;
  double *t0 = ws.t0, *t1 = ws.t1;
  if (op.nmodes == 2) {
    const int nx = op.n[0], ny = op.n[1];
    right_batched(r, (long long)nvec * nx, ny, op.S[1], t0, s);            // R S_y
    GemmArgs g = left(op.ST[0], nx, t0, ny, ny, op.N, t1, nvec);           // S_x^T (R S_y)
    g.epi = EPI_DIVIDE2;
    g.lamM = op.lam[0];
    g.lamN = op.lam[1];
    g.sigma = sigma;
    gemm(g, s);
    gemm(left(op.S[0], nx, t1, ny, ny, op.N, t0, nvec), s);               // S_x (..)
    right_batched(t0, (long long)nvec * nx, ny, op.ST[1], out, s);         // (..) S_y^T
    return;
  }
  const int n0 = op.n[0], n1 = op.n[1], n2 = op.n[2], n3 = op.n[3];
  const long long s23 = (long long)n2 * n3, s123 = (long long)n1 * s23;
  // forward: S^T along y2, y1, x2, x1 (divide fused into the last)
  right_batched(r, (long long)nvec * n0 * n1 * n2, n3, op.S[3], t0, s);
  gemm(left(op.ST[2], n2, t0, n3, n3, s23, t1, nvec * n0 * n1), s);
  gemm(left(op.ST[1], n1, t1, s23, s23, s123, t0, nvec * n0), s);
  {
    GemmArgs g = left(op.ST[0], n0, t0, s123, s123, op.N, t1, nvec);
    g.epi = EPI_DIVIDE4;
    g.lamM = op.lam[0];
    g.lamN = op.lam[1];
    g.lam2 = op.lam[2];
    g.lam3 = op.lam[3];
    g.n2 = n2;
    g.n3 = n3;
    g.sigma = sigma;
    gemm(g, s);
  }
  // backward: S along x1, x2, y1, y2
  gemm(left(op.S[0], n0, t1, s123, s123, op.N, t0, nvec), s);
  gemm(left(op.S[1], n1, t0, s23, s23, s123, t1, nvec * n0), s);
  gemm(left(op.S[2], n2, t1, n3, n3, s23, t0, nvec * n0 * n1), s);
  right_batched(t0, (long long)nvec * n0 * n1 * n2, n3, op.ST[3], out, s);
}

}  // namespace tps
