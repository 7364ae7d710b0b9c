// FP32-arithmetic mode products: the H-apply of the low-precision solver phase and the
// preconditioner of Sec. 4.2, both with FP64 input and output.
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

namespace {
__global__ void k_to_f32(const double *__restrict__ x, float *__restrict__ y, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    y[e] = (float)x[e];
}
}  // namespace

// H-apply with FP32 arithmetic (Eq. tensor_op1D / tensor_op2D as in the FP64 path): psi is
// converted to FP32 once into the workspace, the mode products and the (V - theta) psi
// epilogue run in FP32 on FP32 copies of K and V, and the result is stored in FP64.  Used by
// the low-precision phase of the mixed-precision solver; its error is that of FP32 dot
// products of length n_k (about n_k eps_32 ||K|| |psi|).
void launch_apply_h_f32(const DevOperator &op, const double *psi, double *out, int nvec,
                        const double *theta_dev, double theta, ApplyWorkspace &ws,
                        cudaStream_t s) {
  if (nvec <= 0) return;
  float *p32 = reinterpret_cast<float *>(ws.t0);
  const long long total = (long long)nvec * op.N;
  long long blocks = (total + 255) / 256;
  if (blocks > 152LL * 32) blocks = 152LL * 32;
  count_launch();
  k_to_f32<<<(unsigned)blocks, 256, 0, s>>>(psi, p32, total);
  auto g32 = [&](const GemmArgs &g) { gemm::gemm<float, float, float, double>(g, s); };
  if (op.nmodes == 2) {
    const int nx = op.n[0], ny = op.n[1];
    GemmArgs g = gemm::base_args();
    g.M = nx;
    g.Nc = ny;
    g.batch = nvec;
    g.nphase = 2;
    g.K[0] = nx;
    g.A[0] = {op.Kf[0], nx, 0};
    g.B[0] = {p32, ny, op.N};
    g.K[1] = ny;
    g.A[1] = {p32, ny, op.N};
    g.B[1] = {op.KTf[1], ny, 0};
    g.C = out;
    g.ldc = ny;
    g.bsc = op.N;
    g.epi = gemm::EPI_HAPPLY;
    g.E = {p32, ny, op.N};
    g.V = op.Vf;
    g.ldv = ny;
    g.theta = theta_dev;
    g.theta0 = theta;
    g32(g);
    return;
  }
  const int n0 = op.n[0], n1 = op.n[1], n2 = op.n[2], n3 = op.n[3];
  const long long s23 = (long long)n2 * n3, s123 = (long long)n1 * s23;
  {
    GemmArgs g = gemm::base_args();
    g.M = n2;
    g.Nc = n3;
    g.batch = nvec * n0 * n1;
    g.nphase = 2;
    g.K[0] = n2;
    g.A[0] = {op.Kf[2], n2, 0};
    g.B[0] = {p32, n3, s23};
    g.K[1] = n3;
    g.A[1] = {p32, n3, s23};
    g.B[1] = {op.KTf[3], n3, 0};
    g.C = out;
    g.ldc = n3;
    g.bsc = s23;
    g.epi = gemm::EPI_HAPPLY;
    g.E = {p32, n3, s23};
    g.V = op.Vf;
    g.ldv = n3;
    g.vbs = s23;
    g.vmod = (long long)n0 * n1;
    g.theta = theta_dev;
    g.theta_div = (long long)n0 * n1;
    g.theta0 = theta;
    g32(g);
  }
  {
    GemmArgs g = left(op.Kf[1], n1, p32, s23, s23, s123, out, nvec * n0);
    g.epi = gemm::EPI_ACCUM;
    g32(g);
  }
  {
    GemmArgs g = left(op.Kf[0], n0, p32, s123, s123, op.N, out, nvec);
    g.epi = gemm::EPI_ACCUM;
    g32(g);
  }
}

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
