// FP64 launchers of the mode-product GEMM (gemm_kernel.cuh): the H-apply of Eq.
// tensor_op1D / Eq. tensor_op2D with V and the shift fused into the epilogue, and the
// fast-diagonalisation preconditioner of Sec. 4.2 with the division fused.
//
// GB300 has no FP64 tensor-core path (tcgen05 has no f64 kind), so these run on the
// FP64 FMA pipe, which they keep busy on every active cycle; tile sizes are chosen per
// launch to balance the blocks over the 152 SMs.
#include "gemm_kernel.cuh"

namespace tps {

gemm::TileCache &gemm::tile_cache() {
  static TileCache cache;
  return cache;
}

using gemm::GemmArgs;
using gemm::base_args;
using gemm::left;

namespace {
inline void gemm64(const GemmArgs &g, cudaStream_t s) { gemm::gemm<double, double, double, double>(g, s); }
inline void right64(const double *A, long long rows, int n, const double *B, double *C,
                    cudaStream_t s) {
  gemm::right_chunked<double, double, double, double>(A, rows, n, B, C, s);
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
    g.epi = gemm::EPI_HAPPLY;
    g.E = {psi, ny, op.N};
    g.V = op.V;
    g.ldv = ny;
    g.vbs = 0;
    g.vmod = 1;
    g.theta = theta_dev;
    g.theta_div = 1;
    g.theta0 = theta;
    gemm64(g, s);
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
    g.epi = gemm::EPI_HAPPLY;
    g.E = {psi, n3, s23};
    g.V = op.V;
    g.ldv = n3;
    g.vbs = s23;
    g.vmod = (long long)n0 * n1;
    g.theta = theta_dev;
    g.theta_div = (long long)n0 * n1;
    g.theta0 = theta;
    gemm64(g, s);
  }
  {  // x2 product, accumulated
    GemmArgs g = left(op.K[1], n1, psi, s23, s23, s123, out, nvec * n0);
    g.epi = gemm::EPI_ACCUM;
    gemm64(g, s);
  }
  {  // x1 product, accumulated
    GemmArgs g = left(op.K[0], n0, psi, s123, s123, op.N, out, nvec);
    g.epi = gemm::EPI_ACCUM;
    gemm64(g, s);
  }
}

void launch_apply_prec(const DevOperator &op, const double *r, double *out, int nvec,
                       double sigma, ApplyWorkspace &ws, cudaStream_t s) {
  if (nvec <= 0) return;
  double *t0 = ws.t0, *t1 = ws.t1;
  if (op.nmodes == 2) {
    const int nx = op.n[0], ny = op.n[1];
    right64(r, (long long)nvec * nx, ny, op.S[1], t0, s);                   // R S_y
    GemmArgs g = left(op.ST[0], nx, t0, ny, ny, op.N, t1, nvec);           // S_x^T (R S_y)
    g.epi = gemm::EPI_DIVIDE2;
    g.lamM = op.lam[0];
    g.lamN = op.lam[1];
    g.sigma = sigma;
    gemm64(g, s);
    gemm64(left(op.S[0], nx, t1, ny, ny, op.N, t0, nvec), s);               // S_x (..)
    right64(t0, (long long)nvec * nx, ny, op.ST[1], out, s);                // (..) S_y^T
    return;
  }
  const int n0 = op.n[0], n1 = op.n[1], n2 = op.n[2], n3 = op.n[3];
  const long long s23 = (long long)n2 * n3, s123 = (long long)n1 * s23;
  right64(r, (long long)nvec * n0 * n1 * n2, n3, op.S[3], t0, s);
  gemm64(left(op.ST[2], n2, t0, n3, n3, s23, t1, nvec * n0 * n1), s);
  gemm64(left(op.ST[1], n1, t1, s23, s23, s123, t0, nvec * n0), s);
  {
    GemmArgs g = left(op.ST[0], n0, t0, s123, s123, op.N, t1, nvec);
    g.epi = gemm::EPI_DIVIDE4;
    g.lamM = op.lam[0];
    g.lamN = op.lam[1];
    g.lam2 = op.lam[2];
    g.lam3 = op.lam[3];
    g.n2 = n2;
    g.n3 = n3;
    g.sigma = sigma;
    gemm64(g, s);
  }
  gemm64(left(op.S[0], n0, t1, s123, s123, op.N, t0, nvec), s);
  gemm64(left(op.S[1], n1, t0, s23, s23, s123, t1, nvec * n0), s);
  gemm64(left(op.S[2], n2, t1, n3, n3, s23, t0, nvec * n0 * n1), s);
  right64(t0, (long long)nvec * n0 * n1 * n2, n3, op.ST[3], out, s);
}

}  // namespace tps
