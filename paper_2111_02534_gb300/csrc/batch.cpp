// Batched sweep over independent problems: a small native executor that runs many
// tps_solve instances concurrently on one GPU.
//
// One instance of the sweep (a 1D grid of 128-384 points per coordinate) is too small to
// occupy 152 SMs for most of its kernels, and its outer loop waits on the host a few
// times per iteration.  The executor keeps several instances in flight: `nstreams` host
// threads each own a non-blocking CUDA stream and pull instance indices from a shared
// atomic counter, so while one instance's host loop waits, others' kernels run.  Every
// instance keeps its own context (operators, potential, workspace).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "pdl.cuh"
#include "tps_internal.h"

extern "C" int tps_solve_batch(tps_ctx **ctxs, int ninst, const int *k, int parity, double tol,
                               int block, const tps_solver_opts *opts, double *evals_host,
                               int kstride, double **evecs_dev, tps_stats *stats, int *status,
                               int nstreams) {
  if (!ctxs || ninst < 0 || !k || !evals_host || !evecs_dev || !status || nstreams < 1 ||
      nstreams > 64)
    return TPS_ERR_INVALID_ARG;
  for (int i = 0; i < ninst; ++i)
    if (!ctxs[i] || k[i] < 1 || k[i] > kstride || !evecs_dev[i]) return TPS_ERR_INVALID_ARG;
  if (ninst == 0) return TPS_OK;
  const int device = ctxs[0]->device;
  for (int i = 0; i < ninst; ++i)
    if (ctxs[i]->device != device) return TPS_ERR_INVALID_ARG;
  std::atomic<int> next{0};
  std::atomic<int> cuda_failure{0};
  const int nt = std::min(nstreams, ninst);
  auto worker = [&]() {
    tps::pdl_enabled = nt == 1;  // dependent launches only without concurrent streams
    if (cudaSetDevice(device) != cudaSuccess) {
      cuda_failure = 1;
      return;
    }
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cuda_failure = 1;
      return;
    }
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= ninst) break;
      tps_stats st;
      std::memset(&st, 0, sizeof(st));
      status[i] = tps_solve(ctxs[i], k[i], parity, tol, block, nullptr, 0, opts,
                            evals_host + (long long)i * kstride, evecs_dev[i], &st, s);
      if (stats) stats[i] = st;
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> threads;
  threads.reserve(nt);
  for (int t = 0; t < nt; ++t) threads.emplace_back(worker);
  for (auto &th : threads) th.join();
  if (cuda_failure) return TPS_ERR_CUDA;
  for (int i = 0; i < ninst; ++i)
    if (status[i] != TPS_OK) return status[i];
  return TPS_OK;
}
