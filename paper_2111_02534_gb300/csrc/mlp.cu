// Learned warm start: a small MLP that maps problem parameters and a state index to the
// coefficients of a rank-R separable approximation of that eigenvector, trained on the
// GPU on eigenvectors the solver itself produced (forward, backward and Adam kernels
// here), and the projection / assembly kernels that connect it to the solver's grids.
//
// Network: features (4) -> [Linear, GELU] x 3 (hidden H) -> Linear -> R (px + py) outputs,
// read as C (R x px) and D (R x py).  The predicted state is
//     psi(x, y) = sum_r (sum_a C[r][a] phi_a(x)) (sum_b D[r][b] chi_b(y)),
// phi_a the x-even cosines cos(a pi x / L_x) (a < px) and chi_b the real Fourier modes
// of y (1, cos, sin, cos 2, sin 2, ...; b < py), both continuous functions on [-L, L),
// so one prediction serves any grid.  Training target: the eigenvector's coefficient
// matrix T = Phi^T psi Chi (px x py, Phi / Chi the modes sampled on the grid and
// normalised there).  Loss per sample (sign and scale of an eigenvector are arbitrary):
//     L = 1 - <P, T>^2 / (|P|^2 |T|^2),  P = C^T D.
// GELU is the exact form x Phi(x) = x (1 + erf(x / sqrt 2)) / 2.
//
// Parameter layout (one FP32 buffer): for layer l = 0..3, W_l row-major [in_l][out_l]
// followed by b_l [out_l].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "tps_internal.h"

namespace tps {
namespace mlp {

constexpr int kLayers = 4;  // three hidden layers and the output layer
constexpr int kTile = 32;

__device__ __forceinline__ float gelu(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Y[B][out] = X[B][in] W[in][out] + b, Z = pre-activation kept for the backward pass,
// A = GELU(Z) (act = 1) or Z (act = 0).  W is FP32 or BF16.  32 x 32 output tile per
// CTA, 256 threads, 4 outputs each.
template <typename TW>
__global__ void __launch_bounds__(256)
k_linear_fwd(const float *__restrict__ X, int B, int in, const TW *__restrict__ W,
             const float *__restrict__ bias, int out, int act, float *__restrict__ Z,
             float *__restrict__ A) {
  __shared__ float xs[kTile][kTile + 1];
  __shared__ float ws[kTile][kTile + 1];
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;  // ty in 0..7
  const int r0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < in; k0 += kTile) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int rr = ty + 8 * j;
      const int r = r0 + rr, k = k0 + tx;
      xs[rr][tx] = (r < B && k < in) ? X[(long long)r * in + k] : 0.f;
      const int kk = k0 + rr, c = c0 + tx;
      ws[rr][tx] = (kk < in && c < out) ? (float)W[(long long)kk * out + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kTile; ++k) {
      const float w = ws[k][tx];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = fmaf(xs[ty + 8 * j][k], w, acc[j]);
    }
    __syncthreads();
  }
  const int c = c0 + tx;
  if (c >= out) return;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = r0 + ty + 8 * j;
    if (r >= B) continue;
    const float z = acc[j] + bias[c];
    if (Z) Z[(long long)r * out + c] = z;
    A[(long long)r * out + c] = act ? gelu(z) : z;
  }
}

// dW[in][out] = X^T dZ, db[out] = sum_rows dZ (one CTA column block, all rows).
__global__ void __launch_bounds__(256)
k_linear_wgrad(const float *__restrict__ X, int B, int in, const float *__restrict__ dZ, int out,
               float *__restrict__ dW, float *__restrict__ db) {
  __shared__ float xs[kTile][kTile + 1];
  __shared__ float gs[kTile][kTile + 1];
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  const int i0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  float bacc = 0.f;
  for (int r0 = 0; r0 < B; r0 += kTile) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int rr = ty + 8 * j;
      const int r = r0 + rr;
      xs[rr][tx] = (r < B && i0 + tx < in) ? X[(long long)r * in + i0 + tx] : 0.f;
      gs[rr][tx] = (r < B && c0 + tx < out) ? dZ[(long long)r * out + c0 + tx] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < kTile; ++r) {
      const float g = gs[r][tx];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = fmaf(xs[r][ty + 8 * j], g, acc[j]);
      if (ty == 0 && blockIdx.y == 0) bacc += g;
    }
    __syncthreads();
  }
  const int c = c0 + tx;
  if (c >= out) return;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int i = i0 + ty + 8 * j;
    if (i < in) dW[(long long)i * out + c] = acc[j];
  }
  if (ty == 0 && blockIdx.y == 0) db[c] = bacc;
}

// dX[B][in] = (dZ W^T) [B][in], then (prev_act) dZ_prev = dX * GELU'(Z_prev) in place.
__global__ void __launch_bounds__(256)
k_linear_xgrad(const float *__restrict__ dZ, int B, int out, const float *__restrict__ W, int in,
               const float *__restrict__ Zprev, float *__restrict__ dX) {
  __shared__ float gs[kTile][kTile + 1];
  __shared__ float ws[kTile][kTile + 1];
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  const int r0 = blockIdx.y * kTile, i0 = blockIdx.x * kTile;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int c0 = 0; c0 < out; c0 += kTile) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int rr = ty + 8 * j;
      gs[rr][tx] = (r0 + rr < B && c0 + tx < out) ? dZ[(long long)(r0 + rr) * out + c0 + tx] : 0.f;
      // ws[c][i] = W[i][c]
      ws[tx][rr] = (i0 + rr < in && c0 + tx < out) ? W[(long long)(i0 + rr) * out + c0 + tx] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int c = 0; c < kTile; ++c) {
      const float w = ws[c][tx];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = fmaf(gs[ty + 8 * j][c], w, acc[j]);
    }
    __syncthreads();
  }
  const int i = i0 + tx;
  if (i >= in) return;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = r0 + ty + 8 * j;
    if (r >= B) continue;
    const long long e = (long long)r * in + i;
    dX[e] = acc[j] * (Zprev ? gelu_grad(Zprev[e]) : 1.f);
  }
}

// Per sample: P = C^T D (px x py), loss = 1 - <P,T>^2/(|P|^2 |T|^2), and dL/d(output)
// into G (same layout as the output row: C then D).  One CTA per sample; loss[s] FP64.
__global__ void __launch_bounds__(256)
k_cosine_loss(const float *__restrict__ out, int R, int px, int py, const float *__restrict__ T,
              float *__restrict__ G, double *__restrict__ loss, float inv_batch) {
  extern __shared__ float sh[];
  float *P = sh;                 // px * py
  float *dP = P + px * py;       // px * py
  __shared__ float red[3][8];
  __shared__ float coef[2];
  const int s = blockIdx.x, tid = threadIdx.x;
  const int dout = R * (px + py);
  const float *C = out + (long long)s * dout;
  const float *D = C + R * px;
  const float *Ts = T + (long long)s * px * py;
  float pt = 0.f, pp = 0.f, tt = 0.f;
  for (int e = tid; e < px * py; e += blockDim.x) {
    const int a = e / py, b = e % py;
    float v = 0.f;
    for (int r = 0; r < R; ++r) v = fmaf(C[r * px + a], D[r * py + b], v);
    P[e] = v;
    const float t = Ts[e];
    pt = fmaf(v, t, pt);
    pp = fmaf(v, v, pp);
    tt = fmaf(t, t, tt);
  }
  for (int o = 16; o > 0; o >>= 1) {
    pt += __shfl_down_sync(0xffffffffu, pt, o);
    pp += __shfl_down_sync(0xffffffffu, pp, o);
    tt += __shfl_down_sync(0xffffffffu, tt, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = pt;
    red[1][tid >> 5] = pp;
    red[2][tid >> 5] = tt;
  }
  __syncthreads();
  if (tid == 0) {
    float a = 0.f, b = 0.f, c = 0.f;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      a += red[0][w];
      b += red[1][w];
      c += red[2][w];
    }
    const float den = fmaxf(b * c, 1e-30f);
    loss[s] = 1.0 - (double)a * a / den;
    // dL/dP = (-2 <P,T> T + 2 <P,T>^2 / |P|^2 P) / (|P|^2 |T|^2), averaged over the batch
    coef[0] = -2.f * a / den * inv_batch;
    coef[1] = 2.f * a * a / (den * fmaxf(b, 1e-30f)) * inv_batch;
  }
  __syncthreads();
  for (int e = tid; e < px * py; e += blockDim.x) dP[e] = coef[0] * Ts[e] + coef[1] * P[e];
  __syncthreads();
  float *Gs = G + (long long)s * dout;
  // dC[r][a] = sum_b dP[a][b] D[r][b],  dD[r][b] = sum_a dP[a][b] C[r][a]
  for (int e = tid; e < R * px; e += blockDim.x) {
    const int r = e / px, a = e % px;
    float v = 0.f;
    for (int b = 0; b < py; ++b) v = fmaf(dP[a * py + b], D[r * py + b], v);
    Gs[e] = v;
  }
  for (int e = tid; e < R * py; e += blockDim.x) {
    const int r = e / py, b = e % py;
    float v = 0.f;
    for (int a = 0; a < px; ++a) v = fmaf(dP[a * py + b], C[r * px + a], v);
    Gs[R * px + e] = v;
  }
}

// Adam (Kingma & Ba 2015) on the flat parameter buffer, step t >= 1.
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void k_to_bf16(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// ---------------------------- grid projection / assembly ----------------------------
// Mode value on the grid point j of n on [-L, L): x-even cosines (kind 0) or the real
// Fourier sequence 1, cos 1, sin 1, cos 2, ... (kind 1), unnormalised.
__device__ __forceinline__ double mode_value(int kind, int a, int j, int n) {
  const double t = 2.0 * 3.14159265358979323846 * j / n - 3.14159265358979323846;  // pi x / L
  if (kind == 0 || a == 0) return kind == 0 ? cos(a * t) : 1.0;
  const int f = (a + 1) / 2;
  return (a & 1) ? cos(f * t) : sin(f * t);
}

// Mode matrix M[j][a] (n x na) scaled to unit discrete norm: column norms are computed
// exactly per column by the kernel below, so any n (even the Nyquist-adjacent) is right.
__global__ void k_mode_matrix(int kind, int n, int na, double *__restrict__ M) {
  const int a = blockIdx.x;
  __shared__ double red[256 / 32];
  double ss = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = mode_value(kind, a, j, n);
    M[(long long)j * na + a] = v;
    ss += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  __shared__ double inv;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    inv = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) M[(long long)j * na + a] *= inv;
}

// 2D product modes: K[(i1 n2 + i2)][(a1 q + a2)] = F1[i1][a1] F2[i2][a2] from two unit-norm
// 1D mode matrices (n1 x q, n2 x q), so every column has unit norm again
__global__ void k_mode_kron(const double *__restrict__ F1, int n1, const double *__restrict__ F2,
                            int n2, int q, double *__restrict__ K) {
  const long long qq = (long long)q * q, total = (long long)n1 * n2 * qq;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / qq;
    const int col = (int)(e % qq);
    const int i1 = (int)(row / n2), i2 = (int)(row % n2), a1 = col / q, a2 = col % q;
    K[e] = F1[(long long)i1 * q + a1] * F2[(long long)i2 * q + a2];
  }
}

// U[v][x][b] = sum_y psi[v][x][y] Chi[y][b]  (first mode product of the projection)
__global__ void k_project_y(const double *__restrict__ psi, long long N, int nx, int ny,
                            const double *__restrict__ Chi, int py, double *__restrict__ U,
                            int nvec) {
  const long long total = (long long)nvec * nx * py;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % py);
    const long long vx = e / py;
    const int x = (int)(vx % nx), v = (int)(vx / nx);
    const double *row = psi + (long long)v * N + (long long)x * ny;
    double s = 0.0;
    for (int y = 0; y < ny; ++y) s = fma(row[y], Chi[(long long)y * py + b], s);
    U[e] = s;
  }
}

// T[v][a][b] = sum_x Phi[x][a] U[v][x][b]  (FP32 training target)
__global__ void k_project_x(const double *__restrict__ U, int nx, int py, const double *__restrict__ Phi,
                            int px, float *__restrict__ T, int nvec) {
  const long long total = (long long)nvec * px * py;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e % py);
    const long long va = e / py;
    const int a = (int)(va % px), v = (int)(va / px);
    const double *Uv = U + (long long)v * nx * py;
    double s = 0.0;
    for (int x = 0; x < nx; ++x) s = fma(Phi[(long long)x * px + a], Uv[(long long)x * py + b], s);
    T[e] = (float)s;
  }
}

// Q[v][a][y] = sum_b (C^T D)[a][b] Chi[y][b] from the network output (one thread per
// (v, a, y); the rank-R product is formed on the fly)
__global__ void k_assemble_y(const float *__restrict__ out, int R, int px, int py,
                             const double *__restrict__ Chi, int ny, double *__restrict__ Q,
                             int nvec) {
  const long long total = (long long)nvec * px * ny;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(e % ny);
    const long long va = e / ny;
    const int a = (int)(va % px), v = (int)(va / px);
    const float *C = out + (long long)v * R * (px + py);
    const float *D = C + R * px;
    double s = 0.0;
    for (int b = 0; b < py; ++b) {
      double pab = 0.0;
      for (int r = 0; r < R; ++r) pab = fma((double)C[r * px + a], (double)D[r * py + b], pab);
      s = fma(pab, Chi[(long long)y * py + b], s);
    }
    Q[e] = s;
  }
}

// psi[v][x][y] = sum_a Phi[x][a] Q[v][a][y]
__global__ void k_assemble_x(const double *__restrict__ Q, int px, int ny,
                             const double *__restrict__ Phi, int nx, double *__restrict__ psi,
                             int nvec) {
  const long long N = (long long)nx * ny, total = (long long)nvec * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(e / N);
    const long long xy = e % N;
    const int x = (int)(xy / ny), y = (int)(xy % ny);
    const double *Qv = Q + (long long)v * px * ny;
    double s = 0.0;
    for (int a = 0; a < px; ++a) s = fma(Phi[(long long)x * px + a], Qv[(long long)a * ny + y], s);
    psi[e] = s;
  }
}

}  // namespace mlp
}  // namespace tps

// ------------------------------------ host ------------------------------------
struct tps_ws {
  int device = 0, px = 0, py = 0, R = 0, H = 0;
  int dims[tps::mlp::kLayers + 1] = {0, 0, 0, 0, 0};
  long long woff[tps::mlp::kLayers] = {0, 0, 0, 0}, boff[tps::mlp::kLayers] = {0, 0, 0, 0};
  long long nparam = 0, step = 0;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *wb = nullptr;
  bool wb_valid = false;
  // activations for batches of up to cap rows
  int cap = 0;
  float *A[tps::mlp::kLayers + 1] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  float *Z[tps::mlp::kLayers] = {nullptr, nullptr, nullptr, nullptr};
  float *dZa = nullptr, *dZb = nullptr;
  double *loss = nullptr;
  // grid scratch (mode matrices and intermediate mode products)
  double *scratch = nullptr;
  long long scratch_len = 0;
  double *x0 = nullptr;        // predicted start block of tps_ws_solve
  long long x0_len = 0;
  float *feat = nullptr;       // device features of tps_ws_solve (up to 64 states)
  std::string err;
};

namespace {

using tps::mlp::kLayers;

int ws_error(tps_ws *ws, int code, const std::string &msg) {
  if (ws) ws->err = msg;
  return code;
}

#define WS_CUDA_TRY(ws, expr)                                                         \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess) return ws_error(ws, TPS_ERR_CUDA, std::string(#expr) + ": " + \
                                                             cudaGetErrorString(_e)); \
  } while (0)

unsigned grid_1d(long long n) {
  long long b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152LL * 32) b = 152LL * 32;
  return (unsigned)b;
}

int ensure_batch(tps_ws *ws, int B) {
  if (B <= ws->cap) return TPS_OK;
  for (int l = 0; l <= kLayers; ++l) {
    cudaFree(ws->A[l]);
    ws->A[l] = nullptr;
  }
  for (int l = 0; l < kLayers; ++l) {
    cudaFree(ws->Z[l]);
    ws->Z[l] = nullptr;
  }
  cudaFree(ws->dZa);
  cudaFree(ws->dZb);
  cudaFree(ws->loss);
  ws->dZa = ws->dZb = nullptr;
  ws->loss = nullptr;
  ws->cap = 0;
  int widest = 0;
  for (int l = 0; l <= kLayers; ++l) widest = std::max(widest, ws->dims[l]);
  for (int l = 0; l <= kLayers; ++l)
    WS_CUDA_TRY(ws, cudaMalloc(&ws->A[l], sizeof(float) * (size_t)B * ws->dims[l]));
  for (int l = 0; l < kLayers; ++l)
    WS_CUDA_TRY(ws, cudaMalloc(&ws->Z[l], sizeof(float) * (size_t)B * ws->dims[l + 1]));
  WS_CUDA_TRY(ws, cudaMalloc(&ws->dZa, sizeof(float) * (size_t)B * widest));
  WS_CUDA_TRY(ws, cudaMalloc(&ws->dZb, sizeof(float) * (size_t)B * widest));
  WS_CUDA_TRY(ws, cudaMalloc(&ws->loss, sizeof(double) * (size_t)B));
  ws->cap = B;
  return TPS_OK;
}

int ensure_scratch(tps_ws *ws, long long len) {
  if (len <= ws->scratch_len) return TPS_OK;
  cudaFree(ws->scratch);
  ws->scratch = nullptr;
  ws->scratch_len = 0;
  WS_CUDA_TRY(ws, cudaMalloc(&ws->scratch, sizeof(double) * (size_t)len));
  ws->scratch_len = len;
  return TPS_OK;
}

// forward pass of B rows already in A[0]; bf16: weights from the BF16 copy
void forward(tps_ws *ws, int B, bool bf16, cudaStream_t s) {
  for (int l = 0; l < kLayers; ++l) {
    const int in = ws->dims[l], out = ws->dims[l + 1];
    const dim3 grid((out + 31) / 32, (B + 31) / 32);
    const int act = l < kLayers - 1 ? 1 : 0;
    tps::count_launch();
    if (bf16)
      tps::mlp::k_linear_fwd<__nv_bfloat16><<<grid, 256, 0, s>>>(
          ws->A[l], B, in, ws->wb + ws->woff[l], ws->w + ws->boff[l], out, act, ws->Z[l],
          ws->A[l + 1]);
    else
      tps::mlp::k_linear_fwd<float><<<grid, 256, 0, s>>>(ws->A[l], B, in, ws->w + ws->woff[l],
                                                         ws->w + ws->boff[l], out, act, ws->Z[l],
                                                         ws->A[l + 1]);
  }
}

int isqrt_exact(int p) {
  int q = 0;
  while ((q + 1) * (q + 1) <= p) ++q;
  return q * q == p ? q : -1;
}

// The grid maps of a context as one matrix product psi ~ Phi P Chi^T: psi viewed as an
// nx x ny matrix (1D: n_x x n_y; 2D: (n_x1 n_x2) x (n_y1 n_y2)), Phi nx x px, Chi ny x py.
struct GridMaps {
  int dim = 1, nx = 0, ny = 0, qx = 0, qy = 0;
  long long len = 0;  // doubles of scratch the maps take (Phi, Chi and 2D 1D-factors)
};

int grid_maps(tps_ws *ws, const tps_ctx *ctx, GridMaps *g) {
  if (!ctx->have_grid) return ws_error(ws, TPS_ERR_INVALID_ARG, "grid not set");
  g->dim = ctx->dim;
  if (ctx->dim == 1) {
    g->nx = ctx->n[0];
    g->ny = ctx->n[1];
    if (2 * ws->px > g->nx || ws->py >= g->ny)
      return ws_error(ws, TPS_ERR_INVALID_ARG, "grid too coarse for the model's modes");
    g->len = (long long)g->nx * ws->px + (long long)g->ny * ws->py;
    return TPS_OK;
  }
  g->qx = isqrt_exact(ws->px);
  g->qy = isqrt_exact(ws->py);
  if (g->qx < 1 || g->qy < 1)
    return ws_error(ws, TPS_ERR_INVALID_ARG, "2D grid maps need px and py perfect squares");
  for (int k = 0; k < 4; ++k)
    if ((k < 2 ? g->qx : g->qy) >= ctx->n[k])
      return ws_error(ws, TPS_ERR_INVALID_ARG, "grid too coarse for the model's modes");
  g->nx = ctx->n[0] * ctx->n[1];
  g->ny = ctx->n[2] * ctx->n[3];
  long long f = 0;
  for (int k = 0; k < 4; ++k) f += (long long)ctx->n[k] * (k < 2 ? g->qx : g->qy);
  g->len = (long long)g->nx * ws->px + (long long)g->ny * ws->py + f;
  return TPS_OK;
}

// unit-norm mode matrices: 1D Phi (x-even cosines) and Chi (real Fourier modes); 2D the
// products of the real Fourier modes of the two Cartesian components of x (and of y)
void mode_matrices(tps_ws *ws, const tps_ctx *ctx, const GridMaps &g, double *Phi, double *Chi,
                   cudaStream_t s) {
  if (g.dim == 1) {
    tps::count_launch();
    tps::mlp::k_mode_matrix<<<ws->px, 256, 0, s>>>(0, g.nx, ws->px, Phi);
    tps::count_launch();
    tps::mlp::k_mode_matrix<<<ws->py, 256, 0, s>>>(1, g.ny, ws->py, Chi);
    return;
  }
  double *F = Chi + (long long)g.ny * ws->py, *Fk[4];
  for (int k = 0; k < 4; ++k) {
    const int q = k < 2 ? g.qx : g.qy;
    Fk[k] = F;
    tps::count_launch();
    tps::mlp::k_mode_matrix<<<q, 256, 0, s>>>(1, ctx->n[k], q, F);
    F += (long long)ctx->n[k] * q;
  }
  tps::count_launch();
  tps::mlp::k_mode_kron<<<grid_1d((long long)g.nx * ws->px), 256, 0, s>>>(
      Fk[0], ctx->n[0], Fk[1], ctx->n[1], g.qx, Phi);
  tps::count_launch();
  tps::mlp::k_mode_kron<<<grid_1d((long long)g.ny * ws->py), 256, 0, s>>>(
      Fk[2], ctx->n[2], Fk[3], ctx->n[3], g.qy, Chi);
}

}  // namespace

extern "C" {

int tps_ws_create(tps_ws **out, int device, int px, int py, int rank, int hidden,
                  unsigned long long seed) {
  if (!out || px < 1 || py < 1 || rank < 1 || hidden < 1 || px > 128 || py > 128 || rank > 64 ||
      hidden > 4096)
    return TPS_ERR_INVALID_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return TPS_ERR_CUDA;
  tps_ws *ws = new tps_ws();
  ws->device = device;
  ws->px = px;
  ws->py = py;
  ws->R = rank;
  ws->H = hidden;
  const int d[kLayers + 1] = {4, hidden, hidden, hidden, rank * (px + py)};
  long long off = 0;
  for (int l = 0; l <= kLayers; ++l) ws->dims[l] = d[l];
  for (int l = 0; l < kLayers; ++l) {
    ws->woff[l] = off;
    off += (long long)d[l] * d[l + 1];
    ws->boff[l] = off;
    off += d[l + 1];
  }
  ws->nparam = off;
  // He-style initialisation from a counter-based generator (splitmix64, Box-Muller)
  std::vector<float> h((size_t)off, 0.f);
  uint64_t state = seed;
  auto next = [&]() {
    uint64_t z = (state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  };
  for (int l = 0; l < kLayers; ++l) {
    const double sd = std::sqrt(2.0 / d[l]) * (l == kLayers - 1 ? 0.5 : 1.0);
    for (long long i = 0; i < (long long)d[l] * d[l + 1]; ++i) {
      const double u1 = ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      const double u2 = ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      h[ws->woff[l] + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) *
                                   std::cos(6.283185307179586 * u2));
    }
  }
  bool ok = cudaMalloc(&ws->w, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc(&ws->g, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc(&ws->m, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc(&ws->v, sizeof(float) * off) == cudaSuccess &&
            cudaMalloc(&ws->wb, sizeof(__nv_bfloat16) * off) == cudaSuccess &&
            cudaMemcpy(ws->w, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice) ==
                cudaSuccess &&
            cudaMemset(ws->g, 0, sizeof(float) * off) == cudaSuccess &&
            cudaMemset(ws->m, 0, sizeof(float) * off) == cudaSuccess &&
            cudaMemset(ws->v, 0, sizeof(float) * off) == cudaSuccess &&
            cudaStreamSynchronize(cudaStreamLegacy) == cudaSuccess;
  if (!ok) {
    tps_ws_destroy(ws);
    return TPS_ERR_NOMEM;
  }
  *out = ws;
  return TPS_OK;
}

int tps_ws_destroy(tps_ws *ws) {
  if (!ws) return TPS_ERR_INVALID_ARG;
  cudaSetDevice(ws->device);
  cudaFree(ws->w);
  cudaFree(ws->g);
  cudaFree(ws->m);
  cudaFree(ws->v);
  cudaFree(ws->wb);
  for (int l = 0; l <= kLayers; ++l) cudaFree(ws->A[l]);
  for (int l = 0; l < kLayers; ++l) cudaFree(ws->Z[l]);
  cudaFree(ws->dZa);
  cudaFree(ws->dZb);
  cudaFree(ws->loss);
  cudaFree(ws->scratch);
  cudaFree(ws->x0);
  cudaFree(ws->feat);
  delete ws;
  return TPS_OK;
}

const char *tps_ws_last_error(const tps_ws *ws) { return ws ? ws->err.c_str() : "null model"; }

int tps_ws_info(const tps_ws *ws, long long *nparam, int *out_dim) {
  if (!ws) return TPS_ERR_INVALID_ARG;
  if (nparam) *nparam = ws->nparam;
  if (out_dim) *out_dim = ws->dims[kLayers];
  return TPS_OK;
}

int tps_ws_get_params(tps_ws *ws, float *host, long long n) {
  if (!ws || !host || n != ws->nparam) return TPS_ERR_INVALID_ARG;
  WS_CUDA_TRY(ws, cudaSetDevice(ws->device));
  WS_CUDA_TRY(ws, cudaMemcpy(host, ws->w, sizeof(float) * n, cudaMemcpyDeviceToHost));
  return TPS_OK;
}

int tps_ws_set_params(tps_ws *ws, const float *host, long long n) {
  if (!ws || !host || n != ws->nparam) return TPS_ERR_INVALID_ARG;
  WS_CUDA_TRY(ws, cudaSetDevice(ws->device));
  WS_CUDA_TRY(ws, cudaMemcpy(ws->w, host, sizeof(float) * n, cudaMemcpyHostToDevice));
  WS_CUDA_TRY(ws, cudaStreamSynchronize(cudaStreamLegacy));
  ws->wb_valid = false;
  return TPS_OK;
}

int tps_ws_features(int n, const double *mass_ratio, const double *v0, const double *sigma,
                    const int *state, float *X_host) {
  if (n < 0 || (n > 0 && (!mass_ratio || !v0 || !sigma || !state || !X_host)))
    return TPS_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (!(mass_ratio[i] > 0) || !(v0[i] > 0) || !(sigma[i] > 0) || state[i] < 0)
      return TPS_ERR_INVALID_ARG;
    X_host[4 * i + 0] = (float)(std::log(mass_ratio[i]) / std::log(40.0));
    X_host[4 * i + 1] = (float)(std::log(v0[i]) / 5.0);
    X_host[4 * i + 2] = (float)(std::log(sigma[i]) / std::log(2.0));
    X_host[4 * i + 3] = (float)(state[i] / 8.0);
  }
  return TPS_OK;
}

int tps_ws_forward(tps_ws *ws, const float *X_dev, int B, int bf16, float *out_dev,
                   cudaStream_t stream) {
  if (!ws || B < 0 || (B > 0 && (!X_dev || !out_dev))) return TPS_ERR_INVALID_ARG;
  if (B == 0) return TPS_OK;
  WS_CUDA_TRY(ws, cudaSetDevice(ws->device));
  int st = ensure_batch(ws, B);
  if (st) return st;
  if (bf16 && !ws->wb_valid) {
    tps::count_launch();
    tps::mlp::k_to_bf16<<<grid_1d(ws->nparam), 256, 0, stream>>>(ws->w, ws->wb, ws->nparam);
    ws->wb_valid = true;
  }
  WS_CUDA_TRY(ws, cudaMemcpyAsync(ws->A[0], X_dev, sizeof(float) * 4 * B,
                                  cudaMemcpyDeviceToDevice, stream));
  forward(ws, B, bf16 != 0, stream);
  WS_CUDA_TRY(ws, cudaMemcpyAsync(out_dev, ws->A[kLayers], sizeof(float) * B * ws->dims[kLayers],
                                  cudaMemcpyDeviceToDevice, stream));
  WS_CUDA_TRY(ws, cudaGetLastError());
  return TPS_OK;
}

int tps_ws_loss_grad(tps_ws *ws, const float *X_dev, const float *T_dev, int B, double *loss_host,
                     float *grad_host, cudaStream_t stream) {
  if (!ws || B < 1 || !X_dev || !T_dev) return TPS_ERR_INVALID_ARG;
  WS_CUDA_TRY(ws, cudaSetDevice(ws->device));
  int st = ensure_batch(ws, B);
  if (st) return st;
  WS_CUDA_TRY(ws, cudaMemcpyAsync(ws->A[0], X_dev, sizeof(float) * 4 * B,
                                  cudaMemcpyDeviceToDevice, stream));
  forward(ws, B, false, stream);
  // loss and dL/d(output) into dZa
  const size_t shm = sizeof(float) * 2 * ws->px * ws->py;
  tps::count_launch();
  tps::mlp::k_cosine_loss<<<B, 256, shm, stream>>>(ws->A[kLayers], ws->R, ws->px, ws->py, T_dev,
                                                   ws->dZa, ws->loss, 1.0f / B);
  float *dz = ws->dZa, *dprev = ws->dZb;
  for (int l = kLayers - 1; l >= 0; --l) {
    const int in = ws->dims[l], out = ws->dims[l + 1];
    tps::count_launch();
    tps::mlp::k_linear_wgrad<<<dim3((out + 31) / 32, (in + 31) / 32), 256, 0, stream>>>(
        ws->A[l], B, in, dz, out, ws->g + ws->woff[l], ws->g + ws->boff[l]);
    if (l > 0) {
      tps::count_launch();
      tps::mlp::k_linear_xgrad<<<dim3((in + 31) / 32, (B + 31) / 32), 256, 0, stream>>>(
          dz, B, out, ws->w + ws->woff[l], in, ws->Z[l - 1], dprev);
      std::swap(dz, dprev);
    }
  }
  if (loss_host) {
    std::vector<double> h(B);
    WS_CUDA_TRY(ws, cudaMemcpyAsync(h.data(), ws->loss, sizeof(double) * B,
                                    cudaMemcpyDeviceToHost, stream));
    WS_CUDA_TRY(ws, cudaStreamSynchronize(stream));
    double t = 0.0;
    for (double x : h) t += x;
    *loss_host = t / B;
  }
  if (grad_host) {
    WS_CUDA_TRY(ws, cudaMemcpyAsync(grad_host, ws->g, sizeof(float) * ws->nparam,
                                    cudaMemcpyDeviceToHost, stream));
    WS_CUDA_TRY(ws, cudaStreamSynchronize(stream));
  }
  WS_CUDA_TRY(ws, cudaGetLastError());
  return TPS_OK;
}

int tps_ws_adam_step(tps_ws *ws, float lr, float beta1, float beta2, float eps,
                     cudaStream_t stream) {
  if (!ws || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return TPS_ERR_INVALID_ARG;
  WS_CUDA_TRY(ws, cudaSetDevice(ws->device));
  ws->step += 1;
  const float c1 = 1.f - std::pow(beta1, (float)ws->step);
  const float c2 = 1.f - std::pow(beta2, (float)ws->step);
  tps::count_launch();
  tps::mlp::k_adam<<<grid_1d(ws->nparam), 256, 0, stream>>>(ws->w, ws->g, ws->m, ws->v,
                                                            ws->nparam, lr, beta1, beta2, eps, c1,
                                                            c2);
  ws->wb_valid = false;
  WS_CUDA_TRY(ws, cudaGetLastError());
  return TPS_OK;
}

int tps_ws_project(tps_ws *ws, tps_ctx *ctx, const double *evecs_dev, int k, float *T_dev,
                   cudaStream_t stream) {
  if (!ws || !ctx || k < 0 || (k > 0 && (!evecs_dev || !T_dev))) return TPS_ERR_INVALID_ARG;
  GridMaps g;
  int st = grid_maps(ws, ctx, &g);
  if (st) return st;
  const int nx = g.nx, ny = g.ny;
  if (k == 0) return TPS_OK;
  WS_CUDA_TRY(ws, cudaSetDevice(ws->device));
  st = ensure_scratch(ws, g.len + (long long)k * nx * ws->py);
  if (st) return st;
  double *Phi = ws->scratch, *Chi = Phi + (long long)nx * ws->px, *U = ws->scratch + g.len;
  mode_matrices(ws, ctx, g, Phi, Chi, stream);
  tps::count_launch();
  tps::mlp::k_project_y<<<grid_1d((long long)k * nx * ws->py), 256, 0, stream>>>(
      evecs_dev, (long long)nx * ny, nx, ny, Chi, ws->py, U, k);
  tps::count_launch();
  tps::mlp::k_project_x<<<grid_1d((long long)k * ws->px * ws->py), 256, 0, stream>>>(
      U, nx, ws->py, Phi, ws->px, T_dev, k);
  WS_CUDA_TRY(ws, cudaGetLastError());
  return TPS_OK;
}

int tps_ws_predict(tps_ws *ws, tps_ctx *ctx, const float *X_dev, int k, double *x0_dev,
                   cudaStream_t stream) {
  if (!ws || !ctx || k < 0 || (k > 0 && (!X_dev || !x0_dev))) return TPS_ERR_INVALID_ARG;
  GridMaps g;
  int st = grid_maps(ws, ctx, &g);
  if (st) return st;
  const int nx = g.nx, ny = g.ny;
  if (k == 0) return TPS_OK;
  WS_CUDA_TRY(ws, cudaSetDevice(ws->device));
  st = ensure_batch(ws, k);
  if (st) return st;
  st = ensure_scratch(ws, g.len + (long long)k * ws->px * ny);
  if (st) return st;
  if (!ws->wb_valid) {
    tps::count_launch();
    tps::mlp::k_to_bf16<<<grid_1d(ws->nparam), 256, 0, stream>>>(ws->w, ws->wb, ws->nparam);
    ws->wb_valid = true;
  }
  WS_CUDA_TRY(ws, cudaMemcpyAsync(ws->A[0], X_dev, sizeof(float) * 4 * k,
                                  cudaMemcpyDeviceToDevice, stream));
  forward(ws, k, true, stream);
  double *Phi = ws->scratch, *Chi = Phi + (long long)nx * ws->px, *Q = ws->scratch + g.len;
  mode_matrices(ws, ctx, g, Phi, Chi, stream);
  tps::count_launch();
  tps::mlp::k_assemble_y<<<grid_1d((long long)k * ws->px * ny), 256, 0, stream>>>(
      ws->A[kLayers], ws->R, ws->px, ws->py, Chi, ny, Q, k);
  tps::count_launch();
  tps::mlp::k_assemble_x<<<grid_1d((long long)k * nx * ny), 256, 0, stream>>>(
      Q, ws->px, ny, Phi, nx, x0_dev, k);
  WS_CUDA_TRY(ws, cudaGetLastError());
  return TPS_OK;
}

int tps_ws_solve(tps_ws *ws, tps_ctx *ctx, double mass_ratio, double v0, double sigma, int k,
                 int parity, double tol, int block, const tps_solver_opts *opts,
                 double *evals_host, double *evecs_dev, tps_stats *stats, int *used_warm,
                 cudaStream_t stream) {
  if (used_warm) *used_warm = 0;
  if (!ctx || k < 1 || block < 1) return TPS_ERR_INVALID_ARG;
  if (!ws)  // no model: the cold-started solver
    return tps_solve(ctx, k, parity, tol, block, nullptr, 0, opts, evals_host, evecs_dev, stats,
                     stream);
  if (!ctx->have_grid) return ws_error(ws, TPS_ERR_INVALID_ARG, "grid not set");
  // the whole first block the solver accepts: k wanted pairs plus its guard pairs
  tps_solver_opts o;
  if (opts)
    o = *opts;
  else
    tps_default_opts(&o);
  const int nw = std::min(k + std::max(0, o.guard), 64);
  std::vector<double> mr(nw, mass_ratio), vv(nw, v0), sg(nw, sigma);
  std::vector<int> idx(nw);
  for (int i = 0; i < nw; ++i) idx[i] = i;
  std::vector<float> X(4 * (size_t)nw);
  int st = tps_ws_features(nw, mr.data(), vv.data(), sg.data(), idx.data(), X.data());
  if (st) return ws_error(ws, st, "bad problem parameters");
  WS_CUDA_TRY(ws, cudaSetDevice(ws->device));
  long long N = 1;
  for (int d = 0; d < 2 * ctx->dim; ++d) N *= ctx->n[d];
  if (!ws->feat) WS_CUDA_TRY(ws, cudaMalloc(&ws->feat, sizeof(float) * 4 * 64));
  if (ws->x0_len < (long long)nw * N) {
    cudaFree(ws->x0);
    ws->x0 = nullptr;
    ws->x0_len = 0;
    WS_CUDA_TRY(ws, cudaMalloc(&ws->x0, sizeof(double) * (size_t)nw * N));
    ws->x0_len = (long long)nw * N;
  }
  WS_CUDA_TRY(ws, cudaMemcpyAsync(ws->feat, X.data(), sizeof(float) * X.size(),
                                  cudaMemcpyHostToDevice, stream));
  st = tps_ws_predict(ws, ctx, ws->feat, nw, ws->x0, stream);
  if (st) return st;
  st = tps_solve(ctx, k, parity, tol, block, ws->x0, nw, opts, evals_host, evecs_dev, stats,
                 stream);
  if (st == TPS_ERR_NOT_CONVERGED) {  // fallback: the cold-started solver
    return tps_solve(ctx, k, parity, tol, block, nullptr, 0, opts, evals_host, evecs_dev, stats,
                     stream);
  }
  if (st == TPS_OK && used_warm) *used_warm = 1;
  return st;
}

}  // extern "C"
