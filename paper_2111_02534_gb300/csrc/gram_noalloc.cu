// tps_gram_noalloc: the Gram product G = A^T B without any device allocation.
//
// Some callers cannot call cudaMalloc: programs whose device memory is owned by a
// memory manager that hands out all of it up front (a framework's caching allocator, a
// service with a fixed memory budget), where an allocation behind the manager's back
// can fail or push a co-tenant out of memory.  tps_gram needs a context, and the context
// allocates its scratch buffer; this entry point needs neither.  Its split-row partial
// sums live in a file-scope device array of fixed size that is part of the loaded
// library image, so the call itself never allocates.
//
// The array is shared by every call on a device and keeps the previous call's
// contents; every partial sum is written before it is read, so nothing needs clearing.
// Calls that overlap on the GPU (for example on two streams at once) race on it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "tps_internal.h"

namespace {

constexpr long long kScratchDoubles = 1LL << 17;  // 1 MiB of partial sums per device
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// partial[pb][c][16]: 4x4 block pb of A^T B summed over the rows of chunk c
__global__ void __launch_bounds__(kThreads)
k_gram_partial_noalloc(const double *__restrict__ A, long long lda, int p,
                       const double *__restrict__ B, long long ldb, int q, long long nrows,
                       int nchunk, double *__restrict__ partial) {
  const int c = blockIdx.x, pb = blockIdx.y;
  const int qb = (q + 3) / 4;
  const int i0 = (pb / qb) * 4, j0 = (pb % qb) * 4;
  const long long rows_per = (nrows + nchunk - 1) / nchunk;
  const long long r0 = (long long)c * rows_per;
  const long long r1 = r0 + rows_per < nrows ? r0 + rows_per : nrows;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (long long r = r0 + threadIdx.x; r < r1; r += kThreads) {
    double a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = (i0 + i < p) ? A[(long long)(i0 + i) * lda + r] : 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = (j0 + j < q) ? B[(long long)(j0 + j) * ldb + r] : 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
  __shared__ double red[kThreads / 32][16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double v = acc[i][j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][i * 4 + j] = v;
    }
  __syncthreads();
  if (threadIdx.x < 16) {
    double v = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) v += red[w][threadIdx.x];
    partial[((long long)pb * nchunk + c) * 16 + threadIdx.x] = v;
  }
}

__global__ void k_gram_reduce_noalloc(const double *__restrict__ partial, int p, int q, int nchunk,
                                      double *__restrict__ G, int ldg) {
  const int qb = (q + 3) / 4;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p * q; e += gridDim.x * blockDim.x) {
    const int i = e % p, j = e / p;
    const int pb = (i / 4) * qb + j / 4;
    const double *src = partial + (long long)pb * nchunk * 16 + (i % 4) * 4 + (j % 4);
    double v = 0.0;
    for (int c = 0; c < nchunk; ++c) v += src[(long long)c * 16];
    G[(long long)j * ldg + i] = v;
  }
}

// Per-device set-up, done once per device and CUDA context with that device current: the
// device address of g_noalloc_scratch (in host code the symbol's name is only a host-side
// stand-in, not a device address) and the SM count that sizes the grid.  The cache is keyed
// by the context's unique id as well as the device number, so a cudaDeviceReset, which ends
// the primary context and with it the module that holds the array, is followed by a fresh
// look-up instead of the use of a stale address.
struct ScratchSetup {
  unsigned long long ctx_id = 0;
  double *addr = nullptr;
  int sms = 0;
};
ScratchSetup g_setup[kMaxDevices];
std::mutex g_scratch_mutex;

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current CUDA context (0 if it cannot be read).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
  });
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c ||
      get_id(c, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

cudaError_t scratch_setup(double **addr, int *sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  // 0 when no context is current on this thread yet: the look-up below then binds the
  // device's primary context, and the id is read again after it
  const unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  ScratchSetup &su = g_setup[dev];
  if (!su.addr || id == 0 || su.ctx_id != id) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    su.addr = static_cast<double *>(p);
    su.sms = n > 0 ? n : 1;
    su.ctx_id = current_context_id();
  }
  *addr = su.addr;
  *sms = su.sms;
  return cudaSuccess;
}

}  // namespace

extern "C" int tps_gram_noalloc(const double *A_dev, long long lda, int p, const double *B_dev,
                                long long ldb, int q, long long nrows, double *G_dev, int ldg,
                                cudaStream_t stream) {
  if (p < 1 || q < 1 || p > 64 || q > 64 || nrows < 0 || lda < nrows || ldb < nrows || ldg < p ||
      !G_dev || (nrows > 0 && (!A_dev || !B_dev)))
    return TPS_ERR_INVALID_ARG;
  double *scratch = nullptr;
  int sms = 1;
  if (scratch_setup(&scratch, &sms) != cudaSuccess) return TPS_ERR_CUDA;
  const int npb = ((p + 3) / 4) * ((q + 3) / 4);
  // row chunks: about two CTAs per SM over all 4x4 blocks, at most one per 1024 rows, and
  // never more than the array holds (its capacity is 2^17 / (16 npb) chunks, 32 at
  // p = q = 64)
  long long nchunk = kScratchDoubles / ((long long)npb * 16);
  const long long want = (2LL * sms + npb - 1) / npb;
  const long long maxc = (nrows + 1023) / 1024;
  if (nchunk > want) nchunk = want;
  if (nchunk > maxc) nchunk = maxc;
  if (nchunk < 1) nchunk = 1;
  // each launch's own status (cudaLaunchKernelEx returns it), so that an error left
  // behind by an earlier, unrelated call is neither reported here nor cleared
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nchunk, npb);
  cfg.blockDim = dim3(kThreads);
  cfg.stream = stream;
  tps::count_launch();
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_gram_partial_noalloc, A_dev, lda, p, B_dev, ldb, q,
                                     nrows, (int)nchunk, scratch);
  if (e != cudaSuccess) return TPS_ERR_CUDA;
  cfg.gridDim = dim3((unsigned)((p * q + 255) / 256));
  cfg.blockDim = dim3(256);
  tps::count_launch();
  e = cudaLaunchKernelEx(&cfg, k_gram_reduce_noalloc, (const double *)scratch, p, q, (int)nchunk,
                         G_dev, ldg);
  return e == cudaSuccess ? TPS_OK : TPS_ERR_CUDA;
}
