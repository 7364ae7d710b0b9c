// C ABI of the tps library: context, problem set-up on the host (grid, dense
// second-derivative matrices, their eigendecompositions, potential, parity-folded
// operators, two-body well depth) and the thin wrappers around the device kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "tps_internal.h"

namespace tps {

std::atomic<long long> g_kernel_launches{0};
std::atomic<int> g_autotune{1};

int set_error(tps_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_error(tps_ctx *ctx, cudaError_t e, const char *where) {
  std::string m = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return set_error(ctx, TPS_ERR_NOMEM, m);
  return set_error(ctx, TPS_ERR_CUDA, m);
}

namespace {

const double kPi = 3.14159265358979323846;

// Dense periodic spectral second derivative on n points of [-L, L): the closed form
// of the periodic sinc interpolant's second derivative, scaled from [0, 2pi).
std::vector<double> d2_matrix(int n, double L) {
  std::vector<double> D((size_t)n * n);
  const double h = 2.0 * kPi / n;
  const double scale = (kPi / L) * (kPi / L);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double v;
      if (i == j) {
        v = -kPi * kPi / (3.0 * h * h) - 1.0 / 6.0;
      } else {
        const double s = std::sin((i - j) * h / 2.0);
        const double sgn = ((i - j) % 2 == 0) ? 1.0 : -1.0;
        v = -sgn / (2.0 * s * s);
      }
      D[(size_t)i * n + j] = v * scale;
    }
  return D;
}

// Orthonormal eigenvectors of D2 (real Fourier modes) as the columns of a row-major
// n x n matrix, ordered [1, cos 1, sin 1, .., cos(n/2-1), sin(n/2-1), Nyquist], and
// the wavenumber of each column.
void fourier_basis(int n, std::vector<double> &S, std::vector<int> &kcol) {
  S.assign((size_t)n * n, 0.0);
  kcol.assign(n, 0);
  int c = 0;
  for (int j = 0; j < n; ++j) S[(size_t)j * n + c] = 1.0 / std::sqrt((double)n);
  kcol[c++] = 0;
  for (int k = 1; k < n / 2; ++k) {
    for (int j = 0; j < n; ++j) {
      const double t = 2.0 * kPi * k * j / n;
      S[(size_t)j * n + c] = std::cos(t) * std::sqrt(2.0 / n);
      S[(size_t)j * n + c + 1] = std::sin(t) * std::sqrt(2.0 / n);
    }
    kcol[c] = k;
    kcol[c + 1] = k;
    c += 2;
  }
  for (int j = 0; j < n; ++j) S[(size_t)j * n + c] = ((j % 2) ? -1.0 : 1.0) / std::sqrt((double)n);
  kcol[c] = n / 2;
}

std::vector<double> transpose(const std::vector<double> &A, int n) {
  std::vector<double> T((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) T[(size_t)j * n + i] = A[(size_t)i * n + j];
  return T;
}

struct HostMode {
  int n = 0;
  std::vector<double> K, S, lam;
  std::vector<double> Sinv;  // S^-1 when the eigenbasis is not orthogonal (else empty)
};

// Mode k of the full grid: K = a D2, S = Fourier basis, lam = -a (k pi / L)^2.
HostMode full_mode(int n, double L, double a) {
  HostMode m;
  m.n = n;
  m.K = d2_matrix(n, L);
  for (auto &v : m.K) v *= a;
  std::vector<int> kcol;
  fourier_basis(n, m.S, kcol);
  m.lam.resize(n);
  for (int c = 0; c < n; ++c) {
    const double kk = kcol[c] * kPi / L;
    m.lam[c] = -a * kk * kk;
  }
  return m;
}

// Mode x folded into a heavy-exchange sector (Sec. 5.1, parity selection rule).
// Even sector: reduced index i = 0..n/2, weights w = (1, 2, .., 2, 1), coordinates
// u_i = sqrt(w_i) P_i, operator sqrt(w_i/w_j) (K_ij + K_i,n-j [0 < j < n/2]); the
// eigenvectors are the cosine modes.  Odd sector: i = 1..n/2-1, K_ij - K_i,n-j, sine modes.
HostMode sector_mode(const HostMode &full, int parity, double L, double a) {
  const int n = full.n;
  HostMode m;
  const bool even = parity == TPS_X_EVEN;
  const int nr = even ? n / 2 + 1 : n / 2 - 1;
  const int off = even ? 0 : 1;
  m.n = nr;
  m.K.assign((size_t)nr * nr, 0.0);
  m.S.assign((size_t)nr * nr, 0.0);
  m.lam.assign(nr, 0.0);
  auto w = [&](int i) { return (i == 0 || i == n / 2) ? 1.0 : 2.0; };
  for (int r = 0; r < nr; ++r) {
    const int i = r + off;
    for (int c = 0; c < nr; ++c) {
      const int j = c + off;
      double v = full.K[(size_t)i * n + j];
      if (j != 0 && j != n / 2) v += (even ? 1.0 : -1.0) * full.K[(size_t)i * n + (n - j)];
      if (even) v *= std::sqrt(w(i) / w(j));
      m.K[(size_t)r * nr + c] = v;
    }
  }
  for (int c = 0; c < nr; ++c) {
    const int k = c + off;
    const double kk = k * kPi / L;
    m.lam[c] = -a * kk * kk;
    for (int r = 0; r < nr; ++r) {
      const int i = r + off;
      const double t = 2.0 * kPi * k * i / n;
      double v;
      if (even) {
        const double norm = (k == 0 || k == n / 2) ? (double)n : n / 2.0;
        v = std::sqrt(w(i)) * std::cos(t) / std::sqrt(norm);
      } else {
        v = 2.0 * std::sin(t) / std::sqrt((double)n);
      }
      m.S[(size_t)r * nr + c] = v;
    }
  }
  return m;
}

int upload(tps_ctx *ctx, double **dst, const std::vector<double> &src) {
  TPS_CUDA_TRY(ctx, cudaMalloc((void **)dst, src.size() * sizeof(double)));
  TPS_CUDA_TRY(ctx, cudaMemcpy(*dst, src.data(), src.size() * sizeof(double),
                               cudaMemcpyHostToDevice));
  return TPS_OK;
}

int upload_f32(tps_ctx *ctx, float **dst, const std::vector<double> &src) {
  std::vector<float> f(src.begin(), src.end());
  TPS_CUDA_TRY(ctx, cudaMalloc((void **)dst, f.size() * sizeof(float)));
  TPS_CUDA_TRY(ctx, cudaMemcpy(*dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
  return TPS_OK;
}

int build_operator(tps_ctx *ctx, DevOperator &op, const std::vector<HostMode> &modes,
                   const std::vector<double> *V) {
  free_operator(op);
  op.nmodes = (int)modes.size();
  op.N = 1;
  double lmin = 0.0, lmax = 0.0;
  for (int k = 0; k < op.nmodes; ++k) {
    const HostMode &m = modes[k];
    op.n[k] = m.n;
    op.N *= m.n;
    int st;
    if ((st = upload(ctx, &op.K[k], m.K))) return st;
    if ((st = upload(ctx, &op.KT[k], transpose(m.K, m.n)))) return st;
    // the fast diagonalisation multiplies mode 0 (x) from the left by S^-1, then S, and
    // the last mode from the right by S^-T, then S^T (orthogonal bases: S^T and S); the
    // S slot holds what is applied first from the right / last from the left
    std::vector<double> Sl = m.S, Sr = transpose(m.S, m.n);
    if (!m.Sinv.empty()) {
      if (k == 0) {
        Sr = m.Sinv;
      } else {
        Sl = transpose(m.Sinv, m.n);
      }
    }
    if ((st = upload(ctx, &op.S[k], Sl))) return st;
    if ((st = upload(ctx, &op.ST[k], Sr))) return st;
    if ((st = upload(ctx, &op.lam[k], m.lam))) return st;
    if ((st = upload_f32(ctx, &op.Sf[k], Sl))) return st;
    if ((st = upload_f32(ctx, &op.STf[k], Sr))) return st;
    if ((st = upload_f32(ctx, &op.lamf[k], m.lam))) return st;
    if ((st = upload_f32(ctx, &op.Kf[k], m.K))) return st;
    if ((st = upload_f32(ctx, &op.KTf[k], transpose(m.K, m.n)))) return st;
    op.lam_h[k] = m.lam;
    lmin += *std::min_element(m.lam.begin(), m.lam.end());
    lmax += *std::max_element(m.lam.begin(), m.lam.end());
  }
  op.lam_min_sum = lmin;
  op.lam_max_sum = lmax;
  // the eigenvalue sums of modes 1.. sorted once, for the per-call singularity test
  op.lam_rest.assign(1, 0.0);
  for (int k = 1; k < op.nmodes && !op.lam_rest.empty(); ++k) {
    if (op.lam_rest.size() * op.lam_h[k].size() > (1u << 22)) {
      op.lam_rest.clear();
      break;
    }
    std::vector<double> nx;
    nx.reserve(op.lam_rest.size() * op.lam_h[k].size());
    for (double a : op.lam_rest)
      for (double b : op.lam_h[k]) nx.push_back(a + b);
    op.lam_rest.swap(nx);
  }
  std::sort(op.lam_rest.begin(), op.lam_rest.end());
  TPS_CUDA_TRY(ctx, cudaMalloc((void **)&op.V, op.N * sizeof(double)));
  if (V) {
    TPS_CUDA_TRY(ctx, cudaMemcpy(op.V, V->data(), op.N * sizeof(double), cudaMemcpyHostToDevice));
    int st = upload_f32(ctx, &op.Vf, *V);
    if (st) return st;
  } else {
    TPS_CUDA_TRY(ctx, cudaMemset(op.V, 0, op.N * sizeof(double)));
    TPS_CUDA_TRY(ctx, cudaMalloc((void **)&op.Vf, op.N * sizeof(float)));
    TPS_CUDA_TRY(ctx, cudaMemset(op.Vf, 0, op.N * sizeof(float)));
  }
  // the uploads above go through the legacy default stream, which the solver's
  // non-blocking streams do not wait for: finish them before any kernel can read them
  TPS_CUDA_TRY(ctx, cudaStreamSynchronize(cudaStreamLegacy));
  return TPS_OK;
}

// Mode on the mapped Chebyshev grid: K = a D2 (non-symmetric), D2 = S diag(lam) S^-1.
int chebyshev_mode(int n, double L, double a, HostMode &m, std::vector<double> &pts) {
  m.n = n;
  pts.assign(n, 0.0);
  m.K.assign((size_t)n * n, 0.0);
  m.S.assign((size_t)n * n, 0.0);
  m.Sinv.assign((size_t)n * n, 0.0);
  m.lam.assign(n, 0.0);
  const int st = tps_chebyshev_grid(n, L, pts.data(), m.K.data(), m.lam.data(), m.S.data(),
                                    m.Sinv.data());
  if (st) return st;
  for (auto &v : m.K) v *= a;
  for (auto &v : m.lam) v *= a;
  return TPS_OK;
}

// Mode x of the mapped Chebyshev grid folded into a heavy-exchange sector: the nodes are
// mirror images (x_i = -x_{n-1-i}, none at 0), coordinates u_i = (P_i +- P_{n-1-i}) / sqrt 2
// for i < n/2, operator K_ij +- K_{i, n-1-j}, its own eigen-decomposition.
int chebyshev_sector_mode(const HostMode &full, int parity, HostMode &m) {
  const int n = full.n, nr = n / 2;
  const double sg = parity == TPS_X_EVEN ? 1.0 : -1.0;
  m.n = nr;
  m.K.assign((size_t)nr * nr, 0.0);
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nr; ++j)
      m.K[(size_t)i * nr + j] = full.K[(size_t)i * n + j] + sg * full.K[(size_t)i * n + (n - 1 - j)];
  m.S.assign((size_t)nr * nr, 0.0);
  m.Sinv.assign((size_t)nr * nr, 0.0);
  m.lam.assign(nr, 0.0);
  return real_eig(nr, m.K.data(), m.lam.data(), m.S.data(), m.Sinv.data()) ? TPS_ERR_SINGULAR
                                                                           : TPS_OK;
}

double shape_f(int shape, double xi) {
  return shape == TPS_GAUSS ? std::exp(-xi * xi) : 1.0 / std::pow(1.0 + xi * xi, 3);
}

double grid_x(int n, double L, int j) { return -L + j * (2.0 * L / n); }


int check_ready(tps_ctx *ctx) {
  if (!ctx) return TPS_ERR_INVALID_ARG;
  if (!ctx->have_masses || !ctx->have_grid)
    return set_error(ctx, TPS_ERR_NOT_CONFIGURED, "masses and grid must be set first");
  return TPS_OK;
}

// Preconditioner singularity test against the host copy of the eigenvalues.
bool prec_singular(const DevOperator &op, double theta) {
  // minimum over the Kronecker sum of |lambda_sum - theta|: mode 0 scanned against the
  // sorted sums of the other modes (built with the operator)
  const std::vector<double> &rest = op.lam_rest;
  const double scale = std::max(std::fabs(op.lam_max_sum), std::fabs(op.lam_min_sum));
  double mind = std::numeric_limits<double>::infinity();
  if (!rest.empty()) {
    for (double a : op.lam_h[0]) {
      const double target = theta - a;
      auto it = std::lower_bound(rest.begin(), rest.end(), target);
      if (it != rest.end()) mind = std::min(mind, std::fabs(*it - target));
      if (it != rest.begin()) mind = std::min(mind, std::fabs(*(it - 1) - target));
    }
  } else if (theta < op.lam_min_sum) {
    mind = op.lam_min_sum - theta;
  } else {
    mind = 0.0;  // shift inside the spectrum range of a grid too large to scan: refuse
  }
  return mind < 1e-14 * scale;
}

}  // namespace

void free_operator(DevOperator &op) {
  for (int k = 0; k < 4; ++k) {
    cudaFree(op.K[k]);
    cudaFree(op.KT[k]);
    cudaFree(op.S[k]);
    cudaFree(op.ST[k]);
    cudaFree(op.lam[k]);
    cudaFree(op.Sf[k]);
    cudaFree(op.STf[k]);
    cudaFree(op.lamf[k]);
    cudaFree(op.Kf[k]);
    cudaFree(op.KTf[k]);
    op.K[k] = op.KT[k] = op.S[k] = op.ST[k] = op.lam[k] = nullptr;
    op.Sf[k] = op.STf[k] = op.lamf[k] = op.Kf[k] = op.KTf[k] = nullptr;
    op.lam_h[k].clear();
  }
  op.lam_rest.clear();
  free_tc_operator(op.tc);
  free_tf_operator(op.tf);
  op.tf = nullptr;
  op.tc = nullptr;
  cudaFree(op.V);
  cudaFree(op.Vf);
  op.V = nullptr;
  op.Vf = nullptr;
  op.nmodes = 0;
  op.N = 0;
}

int ensure_apply_workspace(tps_ctx *ctx, long long doubles) {
  if (ctx->ws.capacity >= doubles) return TPS_OK;
  cudaFree(ctx->ws.t0);
  cudaFree(ctx->ws.t1);
  ctx->ws.t0 = ctx->ws.t1 = nullptr;
  ctx->ws.capacity = 0;
  TPS_CUDA_TRY(ctx, cudaMalloc((void **)&ctx->ws.t0, doubles * sizeof(double)));
  TPS_CUDA_TRY(ctx, cudaMalloc((void **)&ctx->ws.t1, doubles * sizeof(double)));
  ctx->ws.capacity = doubles;
  return TPS_OK;
}

int ensure_gram_scratch(tps_ctx *ctx, long long doubles) {
  if (ctx->gscr.capacity >= doubles) return TPS_OK;
  cudaFree(ctx->gscr.partial);
  cudaFree(ctx->gscr.count);
  ctx->gscr.partial = nullptr;
  ctx->gscr.count = nullptr;
  ctx->gscr.capacity = ctx->gscr.ncount = 0;
  // one ticket per 4x4 block: at most one per 16 partial sums
  const long long ncount = doubles / 16 + 1;
  TPS_CUDA_TRY(ctx, cudaMalloc((void **)&ctx->gscr.partial, doubles * sizeof(double)));
  TPS_CUDA_TRY(ctx, cudaMalloc((void **)&ctx->gscr.count, ncount * sizeof(unsigned)));
  TPS_CUDA_TRY(ctx, cudaMemset(ctx->gscr.count, 0, ncount * sizeof(unsigned)));
  TPS_CUDA_TRY(ctx, cudaStreamSynchronize(cudaStreamLegacy));  // see build_operator
  ctx->gscr.capacity = doubles;
  ctx->gscr.ncount = ncount;
  return TPS_OK;
}

// A new potential changes only V: the sector operators already built keep their mode
// matrices, eigenbases and tensor-core digit slices and get the folded V in place.
int refresh_sector_potentials(tps_ctx *ctx) {
  const int ny = ctx->n[1];
  for (int p = TPS_X_EVEN; p <= TPS_X_ODD; ++p) {
    if (!ctx->sect_ready[p]) continue;
    DevOperator &op = ctx->sect[p];
    const int nr = op.n[0], off = (p == TPS_X_EVEN || ctx->grid_kind == 1) ? 0 : 1;
    std::vector<double> V((size_t)nr * ny);
    for (int r = 0; r < nr; ++r)
      for (int j = 0; j < ny; ++j) V[(size_t)r * ny + j] = ctx->V_host[(size_t)(r + off) * ny + j];
    std::vector<float> Vf(V.begin(), V.end());
    TPS_CUDA_TRY(ctx, cudaMemcpy(op.V, V.data(), V.size() * sizeof(double), cudaMemcpyHostToDevice));
    TPS_CUDA_TRY(ctx, cudaMemcpy(op.Vf, Vf.data(), Vf.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  return TPS_OK;
}

int build_sector_operator(tps_ctx *ctx, int parity) {
  if (ctx->sect_ready[parity]) return TPS_OK;
  if (ctx->dim != 1) return set_error(ctx, TPS_ERR_INVALID_ARG, "parity sectors are 1D only");
  const int nx = ctx->n[0], ny = ctx->n[1];
  std::vector<HostMode> modes;
  int off = parity == TPS_X_EVEN ? 0 : 1;
  if (ctx->grid_kind == 1) {
    HostMode fx, fy, sx;
    std::vector<double> px, py;
    int st = chebyshev_mode(nx, ctx->L[0], ctx->a[0], fx, px);
    if (!st) st = chebyshev_mode(ny, ctx->L[1], ctx->a[1], fy, py);
    if (!st) st = chebyshev_sector_mode(fx, parity, sx);
    if (st) return set_error(ctx, st, "eigen-decomposition of the mapped D2 failed");
    modes = {sx, fy};
    off = 0;
  } else {
    HostMode fx = full_mode(nx, ctx->L[0], ctx->a[0]);
    HostMode fy = full_mode(ny, ctx->L[1], ctx->a[1]);
    modes = {sector_mode(fx, parity, ctx->L[0], ctx->a[0]), fy};
  }
  const int nr = modes[0].n;
  std::vector<double> V((size_t)nr * ny);
  for (int r = 0; r < nr; ++r)
    for (int j = 0; j < ny; ++j) V[(size_t)r * ny + j] = ctx->V_host[(size_t)(r + off) * ny + j];
  int st = build_operator(ctx, ctx->sect[parity], modes, &V);
  if (st) return st;
  ctx->sect_ready[parity] = true;
  return TPS_OK;
}

}  // namespace tps

using namespace tps;

extern "C" {

const char *tps_status_string(int status) {
  switch (status) {
    case TPS_OK: return "ok";
    case TPS_ERR_INVALID_ARG: return "invalid argument";
    case TPS_ERR_NOT_CONFIGURED: return "not configured";
    case TPS_ERR_CUDA: return "CUDA error";
    case TPS_ERR_NOMEM: return "out of device memory";
    case TPS_ERR_SINGULAR: return "singular preconditioner shift";
    case TPS_ERR_NOT_CONVERGED: return "not converged";
    case TPS_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

int tps_create(tps_ctx **out, int dim, int device) {
  if (!out || (dim != 1 && dim != 2)) return TPS_ERR_INVALID_ARG;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || device < 0 || device >= count) return TPS_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return TPS_ERR_CUDA;
  tps_ctx *ctx = new (std::nothrow) tps_ctx;
  if (!ctx) return TPS_ERR_NOMEM;
  ctx->dim = dim;
  ctx->device = device;
  // split-row partial sums of the Gram kernels (16 MB; chunk counts adapt to it)
  if (ensure_gram_scratch(ctx, 1LL << 21) != TPS_OK) {
    delete ctx;
    return TPS_ERR_NOMEM;
  }
  *out = ctx;
  return TPS_OK;
}

int tps_destroy(tps_ctx *ctx) {
  if (!ctx) return TPS_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  free_solver_workspace(ctx);
  free_operator(ctx->full);
  for (auto &s : ctx->sect) free_operator(s);
  cudaFree(ctx->ws.t0);
  cudaFree(ctx->ws.t1);
  cudaFree(ctx->gscr.partial);
  cudaFree(ctx->gscr.count);
  delete ctx;
  return TPS_OK;
}

const char *tps_last_error(const tps_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int tps_set_masses(tps_ctx *ctx, double M, double m, double hbar) {
  if (!ctx) return TPS_ERR_INVALID_ARG;
  if (!(M > 0) || !(m > 0) || !(hbar > 0))
    return set_error(ctx, TPS_ERR_INVALID_ARG, "masses and hbar must be positive");
  // mu_x = M/2, mu_y = 2Mm/(2M+m), a_k = -hbar^2 / (2 mu_k)
  ctx->a[0] = -hbar * hbar / M;
  ctx->a[1] = -hbar * hbar * (2.0 * M + m) / (4.0 * M * m);
  ctx->have_masses = true;
  ctx->have_grid = false;  // operators depend on the coefficients: grid must be set again
  return TPS_OK;
}

int tps_set_alpha(tps_ctx *ctx, double alpha) {
  if (!ctx) return TPS_ERR_INVALID_ARG;
  if (!(alpha > 0)) return set_error(ctx, TPS_ERR_INVALID_ARG, "alpha must be positive");
  ctx->a[0] = -1.0 / (1.0 + alpha);
  ctx->a[1] = -(1.0 + 2.0 * alpha) / (4.0 + 4.0 * alpha);
  ctx->have_masses = true;
  ctx->have_grid = false;
  return TPS_OK;
}

int tps_set_grid(tps_ctx *ctx, const int *n, const double *L) {
  if (!ctx || !n || !L) return TPS_ERR_INVALID_ARG;
  if (!ctx->have_masses) return set_error(ctx, TPS_ERR_NOT_CONFIGURED, "set masses first");
  cudaSetDevice(ctx->device);
  const int nm = 2 * ctx->dim;
  for (int k = 0; k < nm; ++k)
    if (n[k] < 4 || n[k] % 2 || n[k] > 8192 || !(L[k] > 0))
      return set_error(ctx, TPS_ERR_INVALID_ARG, "grid sizes must be even in [4, 8192], L > 0");
  if (ctx->dim == 2 && (n[0] != n[1] || n[2] != n[3] || L[0] != L[1] || L[2] != L[3]))
    return set_error(ctx, TPS_ERR_INVALID_ARG, "2D needs equal grids for (x1,x2) and (y1,y2)");
  for (int k = 0; k < nm; ++k) {
    ctx->n[k] = n[k];
    ctx->L[k] = L[k];
  }
  ctx->grid_kind = 0;
  ctx->pts[0].clear();
  ctx->pts[1].clear();
  std::vector<HostMode> modes;
  for (int k = 0; k < nm; ++k) {
    const double a = (ctx->dim == 1) ? ctx->a[k] : ctx->a[k / 2];
    modes.push_back(full_mode(n[k], L[k], a));
  }
  long long N = 1;
  for (int k = 0; k < nm; ++k) N *= n[k];
  ctx->V_host.assign((size_t)N, 0.0);
  ctx->vmax_ok = false;
  int st = build_operator(ctx, ctx->full, modes, &ctx->V_host);
  if (st) return st;
  for (int p = 0; p < 3; ++p) {
    free_operator(ctx->sect[p]);
    ctx->sect_ready[p] = false;
  }
  // preconditioner intermediates for up to 16 vectors per launch (at most 2^27 doubles)
  long long chunk = (1LL << 27) / N;
  chunk = std::max(1LL, std::min(16LL, chunk));
  if ((st = ensure_apply_workspace(ctx, chunk * N))) return st;
  ctx->have_grid = true;
  ctx->have_V = false;
  return TPS_OK;
}

int tps_set_grid_chebyshev(tps_ctx *ctx, const int *n, const double *L) {
  if (!ctx || !n || !L) return TPS_ERR_INVALID_ARG;
  if (!ctx->have_masses) return set_error(ctx, TPS_ERR_NOT_CONFIGURED, "set masses first");
  if (ctx->dim != 1) return set_error(ctx, TPS_ERR_INVALID_ARG, "Chebyshev grids are 1D only");
  for (int k = 0; k < 2; ++k)
    if (n[k] < 4 || n[k] % 2 || n[k] > 1024 || !(L[k] > 0))
      return set_error(ctx, TPS_ERR_INVALID_ARG, "grid sizes must be even in [4, 1024], L > 0");
  cudaSetDevice(ctx->device);
  std::vector<HostMode> modes(2);
  std::vector<double> pts[2];
  for (int k = 0; k < 2; ++k) {
    const int st = chebyshev_mode(n[k], L[k], ctx->a[k], modes[k], pts[k]);
    if (st) return set_error(ctx, st, "eigen-decomposition of the mapped D2 failed");
  }
  for (int k = 0; k < 2; ++k) {
    ctx->n[k] = n[k];
    ctx->L[k] = L[k];
    ctx->pts[k] = pts[k];
  }
  ctx->grid_kind = 1;
  const long long N = (long long)n[0] * n[1];
  ctx->V_host.assign((size_t)N, 0.0);
  ctx->vmax_ok = false;
  int st = build_operator(ctx, ctx->full, modes, &ctx->V_host);
  if (st) return st;
  for (int p = 0; p < 3; ++p) {
    free_operator(ctx->sect[p]);
    ctx->sect_ready[p] = false;
  }
  long long chunk = (1LL << 27) / N;
  chunk = std::max(1LL, std::min(16LL, chunk));
  if ((st = ensure_apply_workspace(ctx, chunk * N))) return st;
  ctx->have_grid = true;
  ctx->have_V = false;
  return TPS_OK;
}

int tps_set_potential(tps_ctx *ctx, const double *V, int on_device) {
  int st = check_ready(ctx);
  if (st) return st;
  ctx->vmax_ok = false;
  if (!V) return set_error(ctx, TPS_ERR_INVALID_ARG, "null potential");
  cudaSetDevice(ctx->device);
  const size_t bytes = ctx->full.N * sizeof(double);
  if (on_device) {
    TPS_CUDA_TRY(ctx, cudaMemcpy(ctx->V_host.data(), V, bytes, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(ctx->V_host.data(), V, bytes);
  }
  TPS_CUDA_TRY(ctx, cudaMemcpy(ctx->full.V, ctx->V_host.data(), bytes, cudaMemcpyHostToDevice));
  {
    std::vector<float> vf(ctx->V_host.begin(), ctx->V_host.end());
    TPS_CUDA_TRY(ctx, cudaMemcpy(ctx->full.Vf, vf.data(), vf.size() * sizeof(float),
                                 cudaMemcpyHostToDevice));
  }
  if (ctx->dim == 1) {
    st = refresh_sector_potentials(ctx);
    if (st) return st;
  }
  TPS_CUDA_TRY(ctx, cudaStreamSynchronize(cudaStreamLegacy));  // uploads complete (see above)
  ctx->have_V = true;
  return TPS_OK;
}

int tps_set_pair_potential(tps_ctx *ctx, int shape, double v0, double sigma) {
  int st = check_ready(ctx);
  if (st) return st;
  ctx->vmax_ok = false;
  if ((shape != TPS_GAUSS && shape != TPS_LORENTZ3) || !(sigma > 0) || !std::isfinite(v0))
    return set_error(ctx, TPS_ERR_INVALID_ARG, "bad shape, sigma or v0");
  std::vector<double> V(ctx->full.N);
  if (ctx->grid_kind == 1) {  // mapped Chebyshev points: evaluated on the host
    const int nx = ctx->n[0], ny = ctx->n[1];
    for (int i = 0; i < nx; ++i)
      for (int j = 0; j < ny; ++j) {
        const double x = ctx->pts[0][i], y = ctx->pts[1][j];
        V[(size_t)i * ny + j] = -v0 * (shape_f(shape, std::fabs(y - 0.5 * x) / sigma) +
                                       shape_f(shape, std::fabs(y + 0.5 * x) / sigma));
      }
  } else if (ctx->dim == 1) {
    // evaluated on the device (a host loop over all grid points costs milliseconds), then
    // kept on the host too for the sector folding
    cudaSetDevice(ctx->device);
    launch_pair_potential_1d(ctx->n[0], ctx->n[1], ctx->L[0], ctx->L[1], shape, v0, sigma,
                             ctx->full.V, ctx->full.Vf, cudaStreamLegacy);
    TPS_CUDA_TRY(ctx, cudaGetLastError());
    TPS_CUDA_TRY(ctx, cudaMemcpy(ctx->V_host.data(), ctx->full.V, ctx->full.N * sizeof(double),
                                 cudaMemcpyDeviceToHost));
    st = refresh_sector_potentials(ctx);
    if (st) return st;
    TPS_CUDA_TRY(ctx, cudaStreamSynchronize(cudaStreamLegacy));
    ctx->have_V = true;
    return TPS_OK;
  } else {
    const int nx = ctx->n[0], ny = ctx->n[2];
    size_t e = 0;
    for (int i1 = 0; i1 < nx; ++i1)
      for (int i2 = 0; i2 < nx; ++i2)
        for (int j1 = 0; j1 < ny; ++j1)
          for (int j2 = 0; j2 < ny; ++j2) {
            const double x1 = grid_x(nx, ctx->L[0], i1), x2 = grid_x(nx, ctx->L[1], i2);
            const double y1 = grid_x(ny, ctx->L[2], j1), y2 = grid_x(ny, ctx->L[3], j2);
            const double dm = std::hypot(y1 - 0.5 * x1, y2 - 0.5 * x2) / sigma;
            const double dp = std::hypot(y1 + 0.5 * x1, y2 + 0.5 * x2) / sigma;
            V[e++] = -v0 * (shape_f(shape, dm) + shape_f(shape, dp));
          }
  }
  return tps_set_potential(ctx, V.data(), 0);
}

int tps_set_autotune(int on) {
  g_autotune.store(on ? 1 : 0);
  return TPS_OK;
}

int tps_get_info(const tps_ctx *ctx, long long *N, double *hnorm_est) {
  if (!ctx || !ctx->have_grid) return TPS_ERR_NOT_CONFIGURED;
  if (N) *N = ctx->full.N;
  if (hnorm_est) {
    double s = 0.0;
    for (int k = 0; k < 2 * ctx->dim; ++k) {
      if (ctx->grid_kind == 1) {  // the mapped grid: spectral radius of a_k D2_k
        double r = 0.0;
        for (double l : ctx->full.lam_h[k]) r = std::max(r, std::fabs(l));
        s += r;
        continue;
      }
      const double h = 2.0 * ctx->L[k] / ctx->n[k];
      const double a = ctx->dim == 1 ? ctx->a[k] : ctx->a[k / 2];
      s += std::fabs(a) * (kPi / h) * (kPi / h);
    }
    if (!ctx->vmax_ok) {  // scanned once per potential
      double vmax = 0.0;
      for (double v : ctx->V_host) vmax = std::max(vmax, std::fabs(v));
      ctx->vmax = vmax;
      ctx->vmax_ok = true;
    }
    *hnorm_est = s + ctx->vmax;
  }
  return TPS_OK;
}

int tps_chebyshev_grid(int n, double L, double *y_host, double *D2_host, double *lam_host,
                       double *S_host, double *Sinv_host) {
  if (n < 2 || n > 1024 || !(L > 0) || !y_host || !D2_host) return TPS_ERR_INVALID_ARG;
  const bool factors = lam_host || S_host || Sinv_host;
  if (factors && !(lam_host && S_host && Sinv_host)) return TPS_ERR_INVALID_ARG;
  // roots of T_n: t_j = cos(theta_j), theta_j = pi - pi (j + 1/2) / n, so 1 - t_j^2 = s_j^2
  // with s_j = sin(pi (j + 1/2) / n) > 0
  std::vector<double> t(n), sn(n), D((size_t)n * n), DD((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    const double a = kPi * (j + 0.5) / n;
    t[j] = -std::cos(a);
    sn[j] = std::sin(a);
    y_host[j] = L * t[j] / sn[j];
  }
  // derivative of the interpolant on first-kind Chebyshev points, closed form:
  // D_ij = (-1)^(i+j) (s_j / s_i) / (t_i - t_j), D_ii = t_i / (2 s_i^2)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      D[(size_t)i * n + j] = (i == j) ? t[i] / (2.0 * sn[i] * sn[i])
                                      : (((i + j) & 1) ? -1.0 : 1.0) * (sn[j] / sn[i]) / (t[i] - t[j]);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const double dik = D[(size_t)i * n + k];
      for (int j = 0; j < n; ++j) DD[(size_t)i * n + j] += dik * D[(size_t)k * n + j];
    }
  // chain rule: dt/dy = s^3 / L, d^2t/dy^2 = -3 t s^4 / L^2
  for (int i = 0; i < n; ++i) {
    const double s2 = sn[i] * sn[i];
    const double tp = s2 * sn[i] / L, tpp = -3.0 * t[i] * s2 * s2 / (L * L);
    for (int j = 0; j < n; ++j)
      D2_host[(size_t)i * n + j] = tp * tp * DD[(size_t)i * n + j] + tpp * D[(size_t)i * n + j];
  }
  if (factors && real_eig(n, D2_host, lam_host, S_host, Sinv_host) != 0) return TPS_ERR_SINGULAR;
  return TPS_OK;
}

int tps_two_body_v0(int dim, double mu_hl, double hbar, double E0, int shape, double sigma, int n,
                    double L, double *v0_out) {
  if ((dim != 1 && dim != 2) || !(mu_hl > 0) || !(hbar > 0) || !(E0 > 0) || !(sigma > 0) ||
      n < 4 || n % 2 || n > 4096 || !(L > 0) || !v0_out ||
      (shape != TPS_GAUSS && shape != TPS_LORENTZ3))
    return TPS_ERR_INVALID_ARG;
  // (T + E0) psi = v0 F psi  <=>  v0 = 1 / lambda_max(F^1/2 (T + E0)^-1 F^1/2).
  // Power iteration; (T + E0)^-1 through the Fourier eigenbasis of T = -hbar^2/(2mu) D2.
  HostMode m = full_mode(n, L, -hbar * hbar / (2.0 * mu_hl));
  const std::vector<double> &S = m.S;
  const std::vector<double> &lam = m.lam;
  const size_t Nt = dim == 1 ? (size_t)n : (size_t)n * n;
  std::vector<double> sq(Nt);
  for (int i = 0; i < n; ++i) {
    const double x = grid_x(n, L, i);
    if (dim == 1) {
      sq[i] = std::sqrt(shape_f(shape, std::fabs(x) / sigma));
    } else {
      for (int j = 0; j < n; ++j) {
        const double y = grid_x(n, L, j);
        sq[(size_t)i * n + j] = std::sqrt(shape_f(shape, std::hypot(x, y) / sigma));
      }
    }
  }
  std::vector<double> v(sq), t(Nt), u(Nt);
  auto apply = [&](const std::vector<double> &in, std::vector<double> &out) {
    for (size_t e = 0; e < Nt; ++e) u[e] = sq[e] * in[e];
    if (dim == 1) {
      for (int c = 0; c < n; ++c) {  // t = S^T u / (lam + E0)
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += S[(size_t)j * n + c] * u[j];
        t[c] = s / (lam[c] + E0);
      }
      for (int j = 0; j < n; ++j) {  // out = S t
        double s = 0.0;
        for (int c = 0; c < n; ++c) s += S[(size_t)j * n + c] * t[c];
        out[j] = sq[j] * s;
      }
    } else {
      // t = S^T U S, divide, out = S t S^T
      std::vector<double> w((size_t)n * n);
      for (int c = 0; c < n; ++c)
        for (int j = 0; j < n; ++j) {
          double s = 0.0;
          for (int i = 0; i < n; ++i) s += S[(size_t)i * n + c] * u[(size_t)i * n + j];
          w[(size_t)c * n + j] = s;
        }
      for (int c = 0; c < n; ++c)
        for (int d = 0; d < n; ++d) {
          double s = 0.0;
          for (int j = 0; j < n; ++j) s += w[(size_t)c * n + j] * S[(size_t)j * n + d];
          t[(size_t)c * n + d] = s / (lam[c] + lam[d] + E0);
        }
      for (int i = 0; i < n; ++i)
        for (int d = 0; d < n; ++d) {
          double s = 0.0;
          for (int c = 0; c < n; ++c) s += S[(size_t)i * n + c] * t[(size_t)c * n + d];
          w[(size_t)i * n + d] = s;
        }
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          double s = 0.0;
          for (int d = 0; d < n; ++d) s += w[(size_t)i * n + d] * S[(size_t)j * n + d];
          out[(size_t)i * n + j] = sq[(size_t)i * n + j] * s;
        }
    }
  };
  double nrm = 0.0;
  for (double a : v) nrm += a * a;
  nrm = std::sqrt(nrm);
  for (double &a : v) a /= nrm;
  std::vector<double> Gv(Nt);
  double lam_est = 0.0, prev = 0.0;
  int stable = 0;
  for (int it = 0; it < 20000; ++it) {
    apply(v, Gv);
    double rq = 0.0, gn = 0.0;
    for (size_t e = 0; e < Nt; ++e) {
      rq += v[e] * Gv[e];
      gn += Gv[e] * Gv[e];
    }
    lam_est = rq;
    gn = std::sqrt(gn);
    double res2 = 0.0;
    for (size_t e = 0; e < Nt; ++e) {
      const double r = Gv[e] - rq * v[e];
      res2 += r * r;
    }
    for (size_t e = 0; e < Nt; ++e) v[e] = Gv[e] / gn;
    // converged when the residual makes the Rayleigh-quotient error negligible
    if (std::sqrt(res2) <= 1e-9 * rq && std::fabs(rq - prev) <= 1e-15 * rq) {
      if (++stable >= 2) break;
    } else {
      stable = 0;
    }
    prev = rq;
  }
  if (!(lam_est > 0)) return TPS_ERR_NOT_CONVERGED;
  *v0_out = 1.0 / lam_est;
  return TPS_OK;
}

int tps_apply_h(tps_ctx *ctx, const void *psi_dev, void *out_dev, int nvec, double theta,
                int dtype, cudaStream_t stream) {
  int st = check_ready(ctx);
  if (st) return st;
  if ((dtype != TPS_F64 && dtype != TPS_F32 && dtype != TPS_F64_TC) || nvec < 0 ||
      (nvec > 0 && (!psi_dev || !out_dev)) || !std::isfinite(theta))
    return set_error(ctx, TPS_ERR_INVALID_ARG, "bad apply_h arguments");
  if (dtype == TPS_F64_TC && ctx->dim == 2)
    for (int k = 0; k < 4; ++k)
      if (ctx->n[k] > 128)
        return set_error(ctx, TPS_ERR_INVALID_ARG, "TPS_F64_TC in 2D needs n <= 128 per mode");
  const char *a = (const char *)psi_dev, *b = (const char *)out_dev;
  const size_t bytes = (size_t)nvec * ctx->full.N * sizeof(double);
  if (nvec > 0 && a < b + bytes && b < a + bytes)
    return set_error(ctx, TPS_ERR_INVALID_ARG, "psi and out overlap");
  if (dtype == TPS_F32) {
    // the FP32 path converts psi into the workspace: at most its capacity per launch
    const long long cap = 2 * ctx->ws.capacity / ctx->full.N;
    for (int v0 = 0; v0 < nvec; v0 += (int)cap) {
      const int nv = (int)std::min<long long>(cap, nvec - v0);
      launch_apply_h_f32(ctx->full, (const double *)psi_dev + (long long)v0 * ctx->full.N,
                         (double *)out_dev + (long long)v0 * ctx->full.N, nv, nullptr, theta,
                         ctx->ws, stream);
    }
  } else if (dtype == TPS_F64_TC) {
    TPS_CUDA_TRY(ctx, launch_apply_h_tc(ctx->full, (const double *)psi_dev, (double *)out_dev,
                                        nvec, nullptr, theta, stream));
  } else {
    launch_apply_h(ctx->full, (const double *)psi_dev, (double *)out_dev, nvec, nullptr, theta,
                   stream);
  }
  TPS_CUDA_TRY(ctx, cudaGetLastError());
  return TPS_OK;
}

int tps_device_status(tps_ctx *ctx) {
  if (!ctx) return TPS_ERR_INVALID_ARG;
  TPS_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  TPS_CUDA_TRY(ctx, cudaDeviceSynchronize());
  int flag = tc_operator_status(ctx->full) | tf_operator_status(ctx->full);
  for (int p = 0; p < 3; ++p) flag |= tc_operator_status(ctx->sect[p]) | tf_operator_status(ctx->sect[p]);
  flag |= update_split_status();
  if (flag < 0) return set_error(ctx, TPS_ERR_CUDA, "reading the device status flag failed");
  if (flag) return set_error(ctx, TPS_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait");
  return TPS_OK;
}

int tps_apply_prec(tps_ctx *ctx, const void *r_dev, void *out_dev, int nvec, double theta,
                   int dtype, cudaStream_t stream) {
  int st = check_ready(ctx);
  if (st) return st;
  if ((dtype != TPS_F64 && dtype != TPS_F32 && dtype != TPS_TF32_TC) || nvec < 0 ||
      (nvec > 0 && (!r_dev || !out_dev)) || !std::isfinite(theta))
    return set_error(ctx, TPS_ERR_INVALID_ARG, "bad apply_prec arguments");
  if (dtype == TPS_TF32_TC) {
    if (!tf_prec_supported(ctx->full) || ctx->grid_kind != 0)
      return set_error(ctx, TPS_ERR_INVALID_ARG,
                       "the TF32 tensor-core preconditioner needs a Fourier grid (2D: every "
                       "mode 4 to 128 points, a multiple of 4)");
    st = ensure_tf_operator(ctx->full);
    if (st) return set_error(ctx, st, "building the TF32 preconditioner operator failed");
  }
  const char *a = (const char *)r_dev, *b = (const char *)out_dev;
  const size_t bytes = (size_t)nvec * ctx->full.N * sizeof(double);
  if (nvec > 0 && a < b + bytes && b < a + bytes)
    return set_error(ctx, TPS_ERR_INVALID_ARG, "r and out overlap");
  if (prec_singular(ctx->full, theta))
    return set_error(ctx, TPS_ERR_SINGULAR, "shift hits the kinetic spectrum");
  // the workspace (allocated by tps_set_grid) bounds the vectors per launch
  const long long cap = ctx->ws.capacity / ctx->full.N;
  if (cap < 1) return set_error(ctx, TPS_ERR_NOT_CONFIGURED, "no preconditioner workspace");
  for (int v0 = 0; v0 < nvec; v0 += (int)cap) {
    const int nv = (int)std::min<long long>(cap, nvec - v0);
    const double *rin = (const double *)r_dev + (long long)v0 * ctx->full.N;
    double *o = (double *)out_dev + (long long)v0 * ctx->full.N;
    if (dtype == TPS_TF32_TC) {
      st = launch_apply_prec_tf32(ctx->full, rin, o, nv, theta, ctx->ws, stream);
      if (st) return set_error(ctx, st, "TF32 preconditioner launch failed");
    } else if (dtype == TPS_F32) {
      launch_apply_prec_f32(ctx->full, rin, o, nv, theta, ctx->ws, stream);
    } else {
      launch_apply_prec(ctx->full, rin, o, nv, theta, ctx->ws, stream);
    }
  }
  TPS_CUDA_TRY(ctx, cudaGetLastError());
  return TPS_OK;
}

int tps_gram(tps_ctx *ctx, const double *A_dev, long long lda, int p, const double *B_dev,
             long long ldb, int q, long long nrows, double *G_dev, int ldg, cudaStream_t stream) {
  if (!ctx) return TPS_ERR_INVALID_ARG;
  if (p < 1 || q < 1 || p > 64 || q > 64 || nrows < 0 || lda < nrows || ldb < nrows || ldg < p ||
      !G_dev || (nrows > 0 && (!A_dev || !B_dev)))
    return set_error(ctx, TPS_ERR_INVALID_ARG, "bad gram arguments");
  launch_gram(A_dev, lda, 0, p, B_dev, ldb, 0, q, nrows, G_dev, ldg, 0, 1, ctx->gscr, stream);
  TPS_CUDA_TRY(ctx, cudaGetLastError());
  return TPS_OK;
}

int tps_gram_tc(tps_ctx *ctx, const double *A_dev, long long lda, int p, const double *B_dev,
                long long ldb, int q, long long nrows, double *G_dev, int ldg, cudaStream_t stream) {
  if (!ctx) return TPS_ERR_INVALID_ARG;
  if (p < 1 || q < 1 || !gram_split_supported(p, q, 1) || nrows < 0 || lda < nrows ||
      ldb < nrows || ldg < p || !G_dev || (nrows > 0 && (!A_dev || !B_dev)))
    return set_error(ctx, TPS_ERR_INVALID_ARG, "bad gram_tc arguments");
  launch_gram_split(A_dev, lda, p, B_dev, ldb, q, nrows, G_dev, ldg, ctx->gscr, stream);
  TPS_CUDA_TRY(ctx, cudaGetLastError());
  return TPS_OK;
}

int tps_block_update(tps_ctx *ctx, const double *A_dev, long long lda, int p, const double *Y_dev,
                     int ldy, int q, double beta, double *C_dev, long long ldc, long long nrows,
                     cudaStream_t stream) {
  if (!ctx) return TPS_ERR_INVALID_ARG;
  if (p < 0 || q < 1 || p > 64 || q > 64 || nrows < 0 || lda < nrows || ldc < nrows || ldy < p ||
      !C_dev || (p > 0 && (!A_dev || !Y_dev)))
    return set_error(ctx, TPS_ERR_INVALID_ARG, "bad block_update arguments");
  launch_update(A_dev, lda, 0, p, Y_dev, ldy, 0, q, 1.0, beta, C_dev, ldc, 0, nrows, 1, stream);
  TPS_CUDA_TRY(ctx, cudaGetLastError());
  return TPS_OK;
}

int tps_block_update_tc(tps_ctx *ctx, const double *A_dev, long long lda, int p,
                        const double *Y_dev, int ldy, int q, double beta, double *C_dev,
                        long long ldc, long long nrows, cudaStream_t stream) {
  if (!ctx) return TPS_ERR_INVALID_ARG;
  if (p < 0 || q < 1 || p > 64 || q > 64 || nrows < 0 || lda < nrows || ldc < nrows || ldy < p ||
      !C_dev || (p > 0 && (!A_dev || !Y_dev)))
    return set_error(ctx, TPS_ERR_INVALID_ARG, "bad block_update arguments");
  launch_update_split(A_dev, lda, 0, p, Y_dev, ldy, 0, q, 1.0, beta, C_dev, ldc, 0, nrows, 1,
                      stream);
  TPS_CUDA_TRY(ctx, cudaGetLastError());
  return TPS_OK;
}

int tps_small_eigh(tps_ctx *ctx, const double *G_dev, int m, int ldg, double *theta_dev,
                   double *Y_dev, int ldy, cudaStream_t stream) {
  if (!ctx) return TPS_ERR_INVALID_ARG;
  if (m < 1 || m > 64 || ldg < m || ldy < m || !G_dev || !theta_dev || !Y_dev)
    return set_error(ctx, TPS_ERR_INVALID_ARG, "bad small_eigh arguments");
  launch_rr_eigh(G_dev, m, ldg, theta_dev, Y_dev, ldy, stream, 0, nullptr, 0.0, nullptr,
                 TPS_RR_MIXED);
  TPS_CUDA_TRY(ctx, cudaGetLastError());
  return TPS_OK;
}

}  // extern "C"
