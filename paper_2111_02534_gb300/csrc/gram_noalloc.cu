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
#include <cuda_runtime.h>

#include <mutex>

#include "tps_internal.h"

namespace {

constexpr long long kScratchDoubles = 1LL << 17;  // 1 MiB of partial sums per device
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// device address of g_noalloc_scratch, looked up once per device
double *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

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

// Device address of the scratch array for the current device (set-up on first use).
cudaError_t scratch_address(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
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
  if (scratch_address(&scratch) != cudaSuccess) return TPS_ERR_CUDA;
  const int npb = ((p + 3) / 4) * ((q + 3) / 4);
  // as many row chunks as the scratch holds (at least 32 for p = q = 64), up to 2 per SM
  long long nchunk = kScratchDoubles / ((long long)npb * 16);
  const long long want = (2LL * 152 + npb - 1) / npb;
  const long long maxc = (nrows + 1023) / 1024;
  if (nchunk > want) nchunk = want;
  if (nchunk > maxc) nchunk = maxc;
  if (nchunk < 1) nchunk = 1;
  tps::count_launch();
  k_gram_partial_noalloc<<<dim3((unsigned)nchunk, npb), kThreads, 0, stream>>>(
      A_dev, lda, p, B_dev, ldb, q, nrows, (int)nchunk, scratch);
  tps::count_launch();
  k_gram_reduce_noalloc<<<(p * q + 255) / 256, 256, 0, stream>>>(scratch, p, q, (int)nchunk,
                                                                 G_dev, ldg);
  return cudaGetLastError() == cudaSuccess ? TPS_OK : TPS_ERR_CUDA;
}
