// FP64-accurate tall-skinny block updates C = beta C + alpha A Y on the tensor cores
// (the Ritz vectors X = V Y and HX = (HV) Y, restarts, and the projections of the
// orthogonalisation in Sec. 4.1).  A is n x p (p <= 64 per pass, column-major, n up to
// millions), Y is p x q with q <= 8 per CTA group.
//
// The products are emulated by error-free digit splitting (the Ozaki scheme: Ozaki,
// Ogita, Oishi & Rump, Numer. Algorithms 59, 2012), as in the H-apply, with digits sized
// for a contraction of at most 64 terms (split_digits.cuh):
//  * row r of A gets the exponent E_r with |A[r][k]| < 2^E_r for all k, column j of
//    alpha Y the exponent F_j; each value becomes the integer |x| 2^(55 - E), truncated,
//    written in seven signed base-256 digits, most significant first;
//  * the digit pairs (i, j) with i + j <= 7 (34 of the 49) are multiplied in BF16 and the
//    pairs of one level l = i + j are summed in one FP32 accumulator, exactly (every
//    partial sum is an integer below 2^23.6 for p <= 64);
//  * the levels are combined in two int64 Horner sums (levels 0-3 and 4-7) and rounded
//    once to FP64 by integer arithmetic.
// The dropped levels l >= 8 weigh at most 131072 p 2^(E_r + F_j - 78) < p 2^-61 2^(E_r +
// F_j) per entry, and the truncation of the operands to 55 bits 2^-55 of the row maximum:
// the result has the accuracy of an FP64 product, 2^-53 max_k |A[r][k]| sum_k |alpha Y[k][j]|
// per entry (row-wise, not element-wise).
//
// The MMA is the warp-level mma.sync m16n8k16 (BF16 in, FP32 out): the output is only
// q <= 8 columns wide, and a tcgen05.mma costs its issuing thread about 45 cycles
// whatever N, while mma.sync m16n8k16 issues every 2 cycles per SM.  The 34 digit products
// per multiply-add then cost less than the one FP64 FMA they replace on GB300's FP64 pipe
// (4 FLOP/clk/SM).  The digit splitting of A runs on the FP32 and integer pipes.
//
// A streams from HBM through shared memory: a producer warp copies 64-row tiles of A (one
// 512-byte cp.async.bulk per column, completing on an mbarrier) into a ring of stages,
// four consumer warps split and multiply them (16 rows each), so that many tiles are in
// flight per SM while the consumers compute.  Every wait is bounded; a wait that gives up
// records it in a device flag (tps_device_status, tps_solve) and the CTA winds down.
// Inputs that the bulk copy cannot address (A, lda or the batch stride not 16-byte
// aligned) and the last partial tile are read directly from global memory.
#include <cuda_bf16.h>

#include <atomic>
#include <mutex>

#include "ozaki_tc.cuh"
#include "split_digits.cuh"
#include "pdl.cuh"
#include "tps_internal.h"

namespace tps {

// Nonzero after a wait of the staged update kernel gave up (read and cleared by
// update_split_status).
__device__ int g_update_split_err = 0;
// staged launches since the flag was last read (no read, no synchronisation, without any)
std::atomic<long long> g_staged_launches{0};

namespace {

using namespace b256;
constexpr int kUKT = 4;         // k tiles of 16 (p <= 64)
constexpr int kWarps = 8;       // consumer warps, 16 rows each
constexpr int kCons = 32 * kWarps;
constexpr int kRows = 16 * kWarps;  // rows per staged tile
constexpr int kColStride = kRows + 4;  // doubles between the columns of a staged tile (4 mod 8:
                                       // the four column pairs a warp reads hit disjoint banks)
constexpr int kMaxStages = 6;
constexpr int kRingBytes = 100 * 1024;  // stages x stage bytes, at least 2 stages
#ifndef TPS_UPD_MINB
#define TPS_UPD_MINB 2  // resident staged CTAs per SM the register allocation aims at
#endif

__device__ __forceinline__ void mma_16816(float (&c)[4], const uint32_t (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

__device__ __forceinline__ void mma_1688(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(b));
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc::smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(tc::smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(bar)) : "memory");
}

struct UpdArgs {
  const double *A;
  long long lda, bsa;
  int p;
  const double *Y;
  int ldy;
  long long bsy;
  int q;
  double alpha, beta;
  double *C;
  long long ldc, bsc, nrows;
  const int *need;
  int stages;     // staged kernel: ring stages
  bool has_beta;  // beta != 0: C is read
};

// One warp: 16 rows (ra = row0 + g, rb = ra + 8) of C's columns j0 .. j0 + 7, with A's
// entry (k, row r of the block) at As[k * cs + r] (r < 16, rows past nrows not read), KT
// k tiles of 16 (the last one as m16n8k8 when it holds at most 8 indices).
// Fragment layout of m16n8k16 (g = lane / 4, c = lane % 4): A regs {row g, k 2c..2c+1},
// {row g+8, k 2c..}, {row g, k 2c+8..}, {row g+8, k 2c+8..}; B regs {k 2c..2c+1, col g},
// {k 2c+8.., col g}; C {row g, col 2c, 2c+1}, {row g+8, ..}.  release() is called once the
// warp has read its last value of As.
template <int KT, int NG, typename Stride, typename Release>
__device__ __forceinline__ void block16(const UpdArgs &g_, const double *As, Stride cs,
                                        long long row0, const uint2 (*Bd)[kUS][kUKT][32],
                                        const unsigned (*Fraw)[8], int j0, double *Cs,
                                        Release release) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, c = lane & 3;
  const int p = g_.p;
  const long long ra = row0 + g, rb = ra + 8;
  const bool va = ra < g_.nrows, vb = rb < g_.nrows;
  // row exponents from the high words: the thread's k values of rows g and g + 8, then
  // across the quad
  const int *Ah = reinterpret_cast<const int *>(As) + 1;
  unsigned ea = 0, eb = 0;
#pragma unroll
  for (int kt = 0; kt < KT; ++kt)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = 16 * kt + 2 * c + (e & 1) + 8 * (e >> 1);
      if (k < p) {
        if (va) ea = max(ea, (unsigned)Ah[2 * (k * cs + g)] & 0x7FF00000u);
        if (vb) eb = max(eb, (unsigned)Ah[2 * (k * cs + g + 8)] & 0x7FF00000u);
      }
    }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    ea = max(ea, __shfl_xor_sync(0xffffffffu, ea, o));
    eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, o));
  }
  ea >>= 20;
  eb >>= 20;
  float acc[NG][kUL][4];
#pragma unroll
  for (int gg = 0; gg < NG; ++gg)
#pragma unroll
    for (int l = 0; l < kUL; ++l)
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[gg][l][t] = 0.f;
#pragma unroll
  for (int kt = 0; kt < KT; ++kt) {
    const bool full16 = kt < KT - 1 || 16 * kt + 8 < p;
    uint32_t af[kUS][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (r >= 2 && !full16) {
#pragma unroll
        for (int i = 0; i < kUS; ++i) af[i][r] = 0u;
        continue;
      }
      const bool v = (r & 1) ? vb : va;
      const int row = g + 8 * (r & 1);
      const int k = 16 * kt + 2 * c + 8 * (r >> 1);
      uint32_t d[kUS];
      digits_pair((v && k < p) ? As[k * cs + row] : 0.0,
                  (v && k + 1 < p) ? As[(k + 1) * cs + row] : 0.0, (r & 1) ? eb : ea, d);
#pragma unroll
      for (int i = 0; i < kUS; ++i) af[i][r] = d[i];
    }
    if (kt == KT - 1) release();
    // the A digit fragments serve every column group of the CTA
#pragma unroll
    for (int gg = 0; gg < NG; ++gg) {
      if (full16) {
#pragma unroll
        for (int j = 0; j < kUS; ++j) {
          const uint2 b = Bd[gg][j][kt][lane];
#pragma unroll
          for (int i = 0; i < kUS; ++i)
            if (i + j < kUL) mma_16816(acc[gg][i + j], af[i], b);
        }
      } else {
#pragma unroll
        for (int j = 0; j < kUS; ++j) {
          const uint32_t b = Bd[gg][j][kt][lane].x;
#pragma unroll
          for (int i = 0; i < kUS; ++i)
            if (i + j < kUL) mma_1688(acc[gg][i + j], af[i][0], af[i][1], b);
        }
      }
    }
  }
  // combine the levels: value = (hi 2^32 + lo) 2^(E + F - 70), hi = levels 0..3, lo =
  // levels 4..7 (Horner in base 256)
#pragma unroll
  for (int gg = 0; gg < NG; ++gg)
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const bool v = (t & 2) ? vb : va;
    const int jl = 2 * c + (t & 1);
    const int j = j0 + 8 * gg + jl;
    if (!v || j >= g_.q) continue;
    long long hi = 0, lo = 0;
#pragma unroll
    for (int l = 0; l < kUL; ++l) {
      const long long dl = (long long)__float2int_rn(acc[gg][l][t]);
      if (l < kUL / 2)
        hi = hi * 256 + dl;
      else
        lo = lo * 256 + dl;
    }
    const unsigned er = (t & 2) ? eb : ea, fr = Fraw[gg][jl];
    const double val =
        (er && fr) ? combine(hi, lo, (int)er - 1022 + (int)fr - 1022) : 0.0;
    double *dst = Cs + (long long)j * g_.ldc + ((t & 2) ? rb : ra);
    *dst = g_.has_beta ? fma(g_.beta, *dst, val) : val;
  }
}

// Digit planes of alpha Y's columns j0 .. j0 + 7 as m16n8k16 B fragments in shared memory,
// and their column exponents; the kCons consumer threads take part.
__device__ __forceinline__ void y_fragments(const UpdArgs &g_, const double *Ys, int j0,
                                            uint2 (*Bd)[kUKT][32], unsigned *Fraw) {
  const int t = threadIdx.x;
  if (t < 128) {
    const int jl = t >> 4, k0 = t & 15, j = j0 + jl;
    unsigned m = 0;
    if (j < g_.q)
#pragma unroll
      for (int k = k0; k < 64; k += 16)
        if (k < g_.p) m = max(m, raw_exp(g_.alpha * Ys[(long long)j * g_.ldy + k]));
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (k0 == 0) Fraw[jl] = m;
  }
  asm volatile("bar.sync 1, %0;" ::"r"(kCons) : "memory");
  if (t < 32 * kUKT) {
    const int kt = t >> 5, lane = t & 31, g = lane >> 2, c = lane & 3;
    const int j = j0 + g;
    float dv[4][kUS];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = 16 * kt + 2 * c + (e & 1) + 8 * (e >> 1);
      const double y = (j < g_.q && k < g_.p) ? g_.alpha * Ys[(long long)j * g_.ldy + k] : 0.0;
      digits7(y, Fraw[g], dv[e]);
    }
#pragma unroll
    for (int i = 0; i < kUS; ++i)
      Bd[i][kt][lane] = make_uint2(pack_bf16(dv[0][i], dv[1][i]), pack_bf16(dv[2][i], dv[3][i]));
  }
  asm volatile("bar.sync 1, %0;" ::"r"(kCons) : "memory");
}

// Direct variant (kCons threads): A read from global memory, 16-row blocks strided over
// the grid.  For inputs the bulk copy cannot address.
template <int KT>
__global__ void __launch_bounds__(kCons)
k_update_split(const __grid_constant__ UpdArgs g_) {
  pdl_entry();
  if (g_.need && *g_.need == 0) return;  // conditional product (decided on the device)
  __shared__ uint2 Bd[1][kUS][kUKT][32];
  __shared__ unsigned Fraw[1][8];
  const int s = blockIdx.y, j0 = blockIdx.z * 8, warp = threadIdx.x >> 5;
  y_fragments(g_, g_.Y + s * g_.bsy, j0, Bd[0], Fraw[0]);
  const double *As = g_.A + s * g_.bsa;
  double *Cs = g_.C + s * g_.bsc;
  const long long nblk = (g_.nrows + 15) >> 4;
  for (long long blk = (long long)blockIdx.x * kWarps + warp; blk < nblk;
       blk += (long long)gridDim.x * kWarps)
    block16<KT, 1>(g_, As + blk * 16, g_.lda, blk * 16, Bd, Fraw, j0, Cs, [] {});
}

// Staged variant (kCons + 32 threads): warps 0..kWarps-1 consume kRows-row tiles of A
// from a ring of g_.stages shared-memory stages (kColStride doubles between columns), the
// last warp fills it with one cp.async.bulk per column.  CTA i takes tiles i, i + gridDim.x,
// ...  The last tile, if partial, is read from global memory by the consumers.
template <int KT, int NG>
__global__ void __launch_bounds__(kCons + 32, NG == 1 ? TPS_UPD_MINB : 1)
k_update_split_staged(const __grid_constant__ UpdArgs g_) {
  pdl_entry();
  if (g_.need && *g_.need == 0) return;
  extern __shared__ __align__(128) double ring[];
  __shared__ uint2 Bd[NG][kUS][kUKT][32];
  __shared__ unsigned Fraw[NG][8];
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
  __shared__ int abort_flag;
  const int s = blockIdx.y, j0 = blockIdx.z * 8 * NG, warp = threadIdx.x >> 5,
            lane = threadIdx.x & 31;
  const int S = g_.stages, p = g_.p;
  const int stage_d = p * kColStride;  // doubles per stage
  const long long ntiles = (g_.nrows + kRows - 1) / kRows;
  const long long nfull = g_.nrows / kRows;
  const double *As = g_.A + s * g_.bsa;
  double *Cs = g_.C + s * g_.bsc;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], kWarps);
    }
    abort_flag = 0;
    tc::fence_barrier_init();
  }
  __syncthreads();
  if (warp == kWarps) {
    // ---- producer: one bulk copy of kRows doubles per column of a full tile, spread over
    // the lanes
    int last[kMaxStages];
    for (int i = 0; i < kMaxStages; ++i) last[i] = -1;
    bool ok = true;
    int it = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const int st = it % S;
      const uint32_t round = (uint32_t)(it / S);
      if (round > 0) {
        bool w = true;
        if (lane == 0) w = tc::mbar_wait(&empty[st], (round - 1) & 1u, &g_update_split_err, 11);
        w = __shfl_sync(0xffffffffu, w ? 1 : 0, 0) != 0;
        if (!w || *((volatile int *)&abort_flag)) {
          ok = false;
          break;
        }
      }
      const bool fulltile = tile < nfull;
      if (lane == 0) {
        if (fulltile)
          tc::mbar_arrive_expect_tx(&full[st], (uint32_t)p * kRows * 8);
        else
          mbar_arrive(&full[st]);  // partial tile: the consumers read global memory
      }
      __syncwarp();
      if (fulltile)
        for (int k = lane; k < p; k += 32)
          bulk_load(ring + st * stage_d + k * kColStride,
                    As + (long long)k * g_.lda + tile * kRows, kRows * 8, &full[st]);
      last[st] = fulltile ? (int)(round & 1u) : -1;
    }
    if (!ok && lane == 0) atomicExch(&abort_flag, 1);
    __syncthreads();
    // after a failed wait anywhere in the CTA, let every copy this warp started land
    // before the CTA exits (the consumers may have stopped before reading them)
    if (lane == 0 && *((volatile int *)&abort_flag))
      for (int i = 0; i < S; ++i)
        if (last[i] >= 0) tc::mbar_wait(&full[i], (uint32_t)last[i], nullptr, 0);
    return;
  }
  // ---- consumers
#pragma unroll
  for (int gg = 0; gg < NG; ++gg) y_fragments(g_, g_.Y + s * g_.bsy, j0 + 8 * gg, Bd[gg], Fraw[gg]);
  int it = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int st = it % S;
    const uint32_t round = (uint32_t)(it / S);
    bool w = tc::mbar_wait(&full[st], round & 1u, &g_update_split_err, 12);
    w = __all_sync(0xffffffffu, w);
    if (!w || *((volatile int *)&abort_flag)) {
      if (lane == 0) atomicExch(&abort_flag, 1);
      break;
    }
    const long long row0 = tile * kRows + 16 * warp;
    auto release = [&] {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    };
    if (tile < nfull)
      block16<KT, NG>(g_, ring + st * stage_d + 16 * warp, kColStride, row0, Bd, Fraw, j0, Cs,
                      release);
    else
      block16<KT, NG>(g_, As + row0, g_.lda, row0, Bd, Fraw, j0, Cs, release);
  }
  __syncthreads();
}

using UpdKernel = void (*)(UpdArgs);
constexpr int kMaxNG = 3;  // column groups of 8 per staged CTA (A split once for all)
const UpdKernel kStagedK[kMaxNG][kUKT] = {
    {k_update_split_staged<1, 1>, k_update_split_staged<2, 1>, k_update_split_staged<3, 1>,
     k_update_split_staged<4, 1>},
    {k_update_split_staged<1, 2>, k_update_split_staged<2, 2>, k_update_split_staged<3, 2>,
     k_update_split_staged<4, 2>},
    {k_update_split_staged<1, 3>, k_update_split_staged<2, 3>, k_update_split_staged<3, 3>,
     k_update_split_staged<4, 3>}};
const UpdKernel kDirectK[kUKT] = {k_update_split<1>, k_update_split<2>, k_update_split<3>,
                                  k_update_split<4>};

int stages_for(int p) {
  const int stage_bytes = p * kColStride * 8;
  int S = kRingBytes / stage_bytes;
  return S < 2 ? 2 : (S > kMaxStages ? kMaxStages : S);
}

struct StagedCfg {
  int sms = 0;
  int per_sm[kMaxNG][65] = {{0}};  // resident staged CTAs per SM by groups and p (0: unknown)
};

// SM count and residency of the staged kernel on the current device (cached per device).
const StagedCfg &staged_cfg(int p, int ng) {
  static StagedCfg cfg[64];
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  std::lock_guard<std::mutex> lock(mu);
  StagedCfg &c = cfg[dev];
  if (c.sms == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    c.sms = n > 0 ? n : 1;
    for (int g = 0; g < kMaxNG; ++g)
      for (int i = 0; i < kUKT; ++i)
        cudaFuncSetAttribute(kStagedK[g][i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * 64 * kColStride * 8);
  }
  if (p >= 1 && p <= 64 && ng >= 1 && ng <= kMaxNG && c.per_sm[ng - 1][p] == 0) {
    int b = 0;
    const size_t smem = (size_t)stages_for(p) * p * kColStride * 8;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kStagedK[ng - 1][(p + 15) / 16 - 1],
                                                  kCons + 32, smem);
    c.per_sm[ng - 1][p] = b > 0 ? b : 1;
  }
  return c;
}

}  // namespace

// Fill the per-device launch configuration of every slab width (occupancy queries and
// attributes), so that later launches, e.g. during stream capture, make no such calls.
void prewarm_update_split() {
  for (int g = 1; g <= kMaxNG; ++g)
    for (int p = 1; p <= 64; ++p) staged_cfg(p, g);
}

void launch_update_split(const double *A, long long lda, long long bsa, int p, const double *Y,
                         int ldy, long long bsy, int q, double alpha, double beta, double *C,
                         long long ldc, long long bsc, long long nrows, int batch, cudaStream_t s,
                         const int *need) {
  if (q <= 0 || batch <= 0 || nrows <= 0) return;
  if (p <= 0) {  // nothing to add: the FP64 path scales C by beta
    launch_update(A, lda, bsa, p, Y, ldy, bsy, q, alpha, beta, C, ldc, bsc, nrows, batch, s,
                  need, false);
    return;
  }
  // p is processed in slabs of 64 rows of Y; the first slab applies beta
  for (int i0 = 0; i0 < p; i0 += 64) {
    UpdArgs g;
    g.A = A + (long long)i0 * lda;
    g.lda = lda;
    g.bsa = bsa;
    g.p = p - i0 < 64 ? p - i0 : 64;
    g.Y = Y + i0;
    g.ldy = ldy;
    g.bsy = bsy;
    g.q = q;
    g.alpha = alpha;
    g.beta = i0 == 0 ? beta : 1.0;
    g.C = C;
    g.ldc = ldc;
    g.bsc = bsc;
    g.nrows = nrows;
    g.need = need;
    g.has_beta = g.beta != 0.0;
    const int kt = (g.p + 15) / 16 - 1;
    const bool aligned = (reinterpret_cast<uintptr_t>(g.A) & 15) == 0 && (lda & 1) == 0 &&
                         (batch == 1 || (bsa & 1) == 0);
    const long long ntiles = (nrows + kRows - 1) / kRows;
    // up to kMaxNG column groups of 8 per CTA: A's digits are formed once for all of them
    // (at one CTA per SM instead of two; measured at 131,584 rows, p = 40: q = 16 in 46 us,
    // q = 24 in 62 us, against ~54 and ~70 us with a CTA per group; wider q takes groups of
    // one, the three-group kernel's spills making q = 32 no faster)
    const int ng = q <= 8 * kMaxNG ? (q + 7) / 8 : 1;
    const StagedCfg &cfg = staged_cfg(g.p, ng);
    count_launch();
    if (aligned && nrows >= kRows) {
      g.stages = stages_for(g.p);
      const long long want = (long long)cfg.sms * cfg.per_sm[ng - 1][g.p];
      const long long gx = ntiles < want ? ntiles : want;
      const size_t smem = (size_t)g.stages * g.p * kColStride * 8;
      g_staged_launches.fetch_add(1, std::memory_order_relaxed);
      launch_pdl(kStagedK[ng - 1][kt], dim3((unsigned)gx, batch, (q + 8 * ng - 1) / (8 * ng)),
                 kCons + 32, smem, s, g);
    } else {
      g.stages = 0;
      const long long blocks = (nrows + kRows - 1) / kRows;
      const long long gx = blocks < cfg.sms * 4LL ? blocks : cfg.sms * 4LL;
      launch_pdl(kDirectK[kt], dim3((unsigned)gx, batch, (q + 7) / 8), kCons, 0, s, g);
    }
  }
}

// Synchronously reads and clears the timed-out-wait flag of the staged update kernel.
int update_split_status() {
  if (g_staged_launches.exchange(0) == 0) return 0;
  int h = 0;
  if (cudaMemcpyFromSymbol(&h, g_update_split_err, sizeof(int)) != cudaSuccess) return -1;
  if (h) {
    const int z = 0;
    if (cudaMemcpyToSymbol(g_update_split_err, &z, sizeof(int)) != cudaSuccess) return -1;
  }
  return h;
}

}  // namespace tps
