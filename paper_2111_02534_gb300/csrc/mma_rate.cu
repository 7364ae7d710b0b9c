// Issue-rate probe for the tensor-core instructions the library uses (a stand-alone
// program, not part of libtps.so): cycles per tcgen05.mma (kind::f16, BF16 in, FP32
// accumulate) issued back to back by one thread with operands resident in shared memory,
// (a) with the level and k-step indices and the descriptors computed per MMA in a
// runtime-bounded loop, (b) fully unrolled with descriptors formed once; and cycles per
// warp-level mma.sync m16n8k16 (BF16 -> FP32) with 4 to 32 warps per SM.  One CTA per SM,
// every wait bounded.  Build and run: python -m paper_2111_02534_gb300.mma_rate
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "ozaki_tc.cuh"

using namespace tps;

namespace {

constexpr int kSmem = 120 * 1024;  // forces one CTA per SM (tensor memory: 512 columns each)

__device__ void fill_operands(uint8_t *sA, uint8_t *sB) {
  uint16_t *a16 = reinterpret_cast<uint16_t *>(sA), *b16 = reinterpret_cast<uint16_t *>(sB);
  for (int i = threadIdx.x; i < 8192; i += blockDim.x) a16[i] = 0x3F80;   // 16 KB of 1.0
  for (int i = threadIdx.x; i < 16384; i += blockDim.x) b16[i] = 0x3F00;  // 32 KB of 0.5
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// (a): runtime M, N, L; per MMA a level index, a k-step index and two descriptors
__global__ void __launch_bounds__(128, 1) k_loop(int M, int N, int L, int iters, long long *out,
                                                 int *err) {
  extern __shared__ uint8_t raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = base, *sB = base + 16384;
  __shared__ uint64_t bar;
  __shared__ uint32_t holder;
  fill_operands(sA, sB);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
  }
  if (warp == 2) tc::tmem_alloc(&holder, 512);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = holder;
  if (warp == 1 && lane == 0) {
    const uint32_t idesc = tc::idesc_bf16_f32(M, N);
    const uint32_t ab = tc::smem_addr(sA), bb = tc::smem_addr(sB);
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
      const int l = it % L, kk = (it / L) & 3;
      tc::mma_bf16(tmem + (uint32_t)(l * N), tc::smem_desc_sw128(ab + kk * 32),
                   tc::smem_desc_sw128(bb + kk * 32), idesc, it >= L ? 1u : 0u);
    }
    tc::mma_commit(&bar);
    const bool ok = tc::mbar_wait(&bar, 0, err, 1);
    out[blockIdx.x] = ok ? clock64() - t0 : -1;
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 2) tc::tmem_dealloc(tmem, 512);
}

// (b): compile-time M, N, L; the pair loop unrolled, descriptors formed once
template <int M, int N, int L>
__global__ void __launch_bounds__(128, 1) k_unrolled(int reps, long long *out, int *err) {
  extern __shared__ uint8_t raw[];
  uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  uint8_t *sA = base, *sB = base + 16384;
  __shared__ uint64_t bar;
  __shared__ uint32_t holder;
  fill_operands(sA, sB);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
  }
  if (warp == 2) tc::tmem_alloc(&holder, 512);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = holder;
  if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = tc::idesc_bf16_f32(M, N);
    const uint64_t ad = tc::smem_desc_sw128(tc::smem_addr(sA));
    const uint64_t bd = tc::smem_desc_sw128(tc::smem_addr(sB));
    const long long t0 = clock64();
    for (int r = 0; r < reps; ++r) {
#pragma unroll
      for (int l = 0; l < L; ++l)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          tc::mma_bf16(tmem + (uint32_t)(l * N), ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2),
                       idesc, (r | kk) ? 1u : 0u);
    }
    tc::mma_commit(&bar);
    const bool ok = tc::mbar_wait(&bar, 0, err, 1);
    out[blockIdx.x] = ok ? clock64() - t0 : -1;
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 2) tc::tmem_dealloc(tmem, 512);
}

__global__ void k_sync(const uint32_t *in, int iters, long long *out, float *sink) {
  const int t = threadIdx.x;
  const uint32_t a0 = in[t & 63], a1 = in[(t + 1) & 63], a2 = in[(t + 2) & 63],
                 a3 = in[(t + 3) & 63], b0 = in[(t + 4) & 63], b1 = in[(t + 5) & 63];
  float c[8][4];
  for (int j = 0; j < 8; ++j)
    for (int q = 0; q < 4; ++q) c[j][q] = 0.f;
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
          "{%8,%9}, {%0,%1,%2,%3};"
          : "+f"(c[j][0]), "+f"(c[j][1]), "+f"(c[j][2]), "+f"(c[j][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
  for (int j = 0; j < 8; ++j)
    for (int q = 0; q < 4; ++q) s += c[j][q];
  if (s == 12345.f) sink[0] = s;
  if (t == 0) out[blockIdx.x] = t1 - t0;
}

bool check(cudaError_t e) {
  if (e != cudaSuccess) {
    std::printf("CUDA error: %s\n", cudaGetErrorString(e));
    return false;
  }
  return true;
}

long long max_of(const long long *dev) {
  std::vector<long long> h(152);
  cudaMemcpy(h.data(), dev, 152 * sizeof(long long), cudaMemcpyDeviceToHost);
  long long m = 0;
  for (long long v : h) m = v > m ? v : m;
  return m;
}

template <int M, int N, int L>
bool run_unrolled(long long *out, int *err) {
  const int reps = 100;
  if (!check(cudaFuncSetAttribute(k_unrolled<M, N, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem)))
    return false;
  for (int rep = 0; rep < 2; ++rep) {
    k_unrolled<M, N, L><<<152, 128, kSmem>>>(reps, out, err);
    if (!check(cudaDeviceSynchronize())) return false;
  }
  const double cyc = (double)max_of(out) / (reps * L * 4);
  std::printf("tcgen05 unrolled     M=%3d N=%3d: %6.1f cycles/MMA %6.0f FLOP/clk/SM\n", M, N, cyc,
              2.0 * M * N * 16 / cyc);
  return true;
}

}  // namespace

int main() {
  long long *out;
  int *err;
  float *sink;
  uint32_t *in;
  if (!check(cudaMalloc(&out, 152 * sizeof(long long))) || !check(cudaMalloc(&err, sizeof(int))) ||
      !check(cudaMalloc(&sink, sizeof(float))) || !check(cudaMalloc(&in, 64 * sizeof(uint32_t))))
    return 1;
  cudaMemset(err, 0, sizeof(int));
  std::vector<uint32_t> h(64, 0x3F803F80u);
  cudaMemcpy(in, h.data(), 64 * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (!check(cudaFuncSetAttribute(k_loop, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem)))
    return 1;
  const int shapes[][3] = {{128, 16, 10}, {128, 48, 10}, {128, 128, 4}, {128, 256, 2}, {64, 8, 10}};
  for (const auto &c : shapes) {
    for (int rep = 0; rep < 2; ++rep) {
      k_loop<<<152, 128, kSmem>>>(c[0], c[1], c[2], 4000, out, err);
      if (!check(cudaDeviceSynchronize())) return 1;
    }
    const double cyc = (double)max_of(out) / 4000;
    std::printf("tcgen05 runtime loop M=%3d N=%3d: %6.1f cycles/MMA %6.0f FLOP/clk/SM\n", c[0],
                c[1], cyc, 2.0 * c[0] * c[1] * 16 / cyc);
  }
  if (!run_unrolled<128, 16, 10>(out, err) || !run_unrolled<128, 48, 10>(out, err) ||
      !run_unrolled<128, 64, 8>(out, err) || !run_unrolled<128, 96, 5>(out, err) ||
      !run_unrolled<128, 128, 4>(out, err) || !run_unrolled<128, 256, 2>(out, err) ||
      !run_unrolled<64, 8, 10>(out, err))
    return 1;
  for (int warps : {4, 8, 16, 32}) {
    k_sync<<<152, warps * 32>>>(in, 2000, out, sink);
    if (!check(cudaDeviceSynchronize())) return 1;
    const double inst = (double)warps * 2000 * 8;
    const long long cyc = max_of(out);
    std::printf("mma.sync m16n8k16    %2d warps/SM: %5.2f cycles per warp instruction per SM, %6.0f FLOP/clk/SM\n",
                warps, cyc / inst, inst * 4096 / cyc);
  }
  int herr = 0;
  cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
  std::printf("timed-out waits: %d\n", herr);
  return herr ? 2 : 0;
}
