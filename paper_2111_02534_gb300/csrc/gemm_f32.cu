// Preconditioner of Sec. 4.2 with FP32 arithmetic (FP64 input and output).
//
// The preconditioner is an approximation by construction (V is neglected), so its
// mode products need not be FP64: the GMRES correction solve only asks it to be a fixed
// linear operator close to (T - sigma)^-1, and FP32 rounding (~6e-8 relative per
// product, amplified at most by the condition of T - sigma) is far below that need.
// GB300 runs FP32 FMAs 64x faster than FP64 ones.  The first pass reads the FP64
// residual and converts on load, the last pass converts on store; the intermediates are
// FP32 in the FP64 workspace buffers (half their capacity).
#include "gemm_kernel.cuh"

namespace tps {

using gemm::GemmArgs;
using gemm::left;

void launch_apply_prec_f32(const DevOperator &op, const double *r, double *out, int nvec,
                           double sigma, ApplyWorkspace &ws, cudaStream_t s) {
  if (nvec <= 0) return;
  float *t0 = reinterpret_cast<float *>(ws.t0), *t1 = reinterpret_cast<float *>(ws.t1);
  auto g32 = [&](const GemmArgs &g) { gemm::gemm<float, float, float, float>(g, s); };
  if (op.nmodes == 2) {
    const int nx = op.n[0], ny = op.n[1];
    gemm::right_chunked<float, double, float, float>(r, (long long)nvec * nx, ny, op.Sf[1], t0, s);
    GemmArgs g = left(op.STf[0], nx, t0, ny, ny, op.N, t1, nvec);
    g.epi = gemm::EPI_DIVIDE2;
    g.lamM = op.lamf[0];
    g.lamN = op.lamf[1];
    g.sigma = sigma;
    g32(g);
    g32(left(op.Sf[0], nx, t1, ny, ny, op.N, t0, nvec));
    gemm::right_chunked<float, float, float, double>(t0, (long long)nvec * nx, ny, op.STf[1], out, s);
    return;
  }
  const int n0 = op.n[0], n1 = op.n[1], n2 = op.n[2], n3 = op.n[3];
  const long long s23 = (long long)n2 * n3, s123 = (long long)n1 * s23;
  gemm::right_chunked<float, double, float, float>(r, (long long)nvec * n0 * n1 * n2, n3, op.Sf[3],
                                                   t0, s);
  g32(left(op.STf[2], n2, t0, n3, n3, s23, t1, nvec * n0 * n1));
  g32(left(op.STf[1], n1, t1, s23, s23, s123, t0, nvec * n0));
  {
    GemmArgs g = left(op.STf[0], n0, t0, s123, s123, op.N, t1, nvec);
    g.epi = gemm::EPI_DIVIDE4;
    g.lamM = op.lamf[0];
    g.lamN = op.lamf[1];
    g.lam2 = op.lamf[2];
    g.lam3 = op.lamf[3];
    g.n2 = n2;
    g.n3 = n3;
    g.sigma = sigma;
    g32(g);
  }
  g32(left(op.Sf[0], n0, t1, s123, s123, op.N, t0, nvec));
  g32(left(op.Sf[1], n1, t0, s23, s23, s123, t1, nvec * n0));
  g32(left(op.Sf[2], n2, t1, n3, n3, s23, t0, nvec * n0 * n1));
  gemm::right_chunked<float, float, float, double>(t0, (long long)nvec * n0 * n1 * n2, n3,
                                                   op.STf[3], out, s);
}

}  // namespace tps
