// The preconditioner of Sec. 4.2 (Eq. sylvester_equation by fast diagonalisation, 1D) with
// its four mode products on the tcgen05 tensor cores in TF32:
//   t0 = r S_y,  t1 = (S_x^T t0) ./ (lambda_x + lambda_y - sigma),  t2 = S_x t1,  out = t2 S_y^T
// per vector.  The preconditioner only has to be a fixed operator close to (T - sigma)^-1
// inside GMRES, whose corrections are solved to 1e-3; TF32 (10 explicit mantissa bits,
// FP32 accumulation) changes its result by ~2.5e-3 relative (four products, measured on
// an emulation of the truncated inputs), and runs at a multiple of the FP32 pipe's rate.
//
// Every pass is C = A B^T with both operands K-major (K contiguous), which TMA loads as
// 128-byte-swizzled tiles of 32 FP32 values along K: the epilogues of passes 1 and 3
// store transposed (coalesced: a thread owns a row of the accumulator), so that the next
// pass reads its contraction index contiguously.  Rows whose length is not a multiple of 4
// floats (the x-even sector has n_x = n/2 + 1) are padded to one, as TMA strides must be
// multiples of 16 bytes; padding is never read (the tensor maps stop at the true K).
#include <mutex>

#include "fp_convert.cuh"
#include "ozaki_tc.cuh"
#include "pdl.cuh"
#include "tps_internal.h"

namespace tps {
namespace {

// Tiles are 128 x BN with BN a multiple of 16 up to 128, chosen per operator axis
// (tile_n): a tcgen05.mma costs its issuing thread max(~45, N/2) cycles, so tiles of 64 to
// 128 columns keep each MMA useful, while a pass, a short K loop per CTA, is latency-bound
// and gets faster when its tiles fill one wave on the SMs.
constexpr int kBM = 128, kBNMax = 128, kBK = 32;  // K block: 32 FP32 = one 128-byte row
constexpr int kThreads = 128;
constexpr uint32_t kATile = kBM * kBK * 4;        // 16 KB

// Pipeline depth, widest tile, tensor-memory columns and resident CTAs per SM of a pass.
// kIntCvt: the FP64 output's conversions on the integer pipes (fp_convert.cuh), which pays
// in the streaming 2D passes and costs latency in the short 1D ones.
template <int STAGES, int BNMAX, int TMEMC, int MINB, bool INTCVT>
struct TfCfg {
  static constexpr int kStages = STAGES, kBNMax = BNMAX, kTmemCols = TMEMC, kMinBlocks = MINB;
  static constexpr bool kIntCvt = INTCVT;
  static constexpr uint32_t kBTile = (uint32_t)BNMAX * kBK * 4;
  static constexpr size_t kSmem = 1024 + (size_t)STAGES * (kATile + kBTile) + 256;
  static_assert(BNMAX <= TMEMC && MINB * TMEMC <= 512, "tensor memory of the resident CTAs");
};
// 1D passes: K up to the grid size (a deep ring), tiles up to 128 columns, one CTA per SM
using Cfg1 = TfCfg<6, kBNMax, 256, 1, false>;
// 2D passes: K <= 128 (at most four K blocks) and tiles up to 64 columns; four CTAs per SM
// (50 KB of shared memory and 64 tensor-memory columns each) keep four tiles' loads and
// epilogues in flight, the latency a one-CTA pass of short tiles waits on
using Cfg2 = TfCfg<2, 64, 64, 4, true>;

struct TfArgs {
  int M, N, K;
  int BN;                       // tile width (multiple of 16, <= 256; the B box height)
  int R;                        // rows per vector: row m = v R + r
  long long os_v, os_r, os_n;   // output element (v, r, n) at v os_v + r os_r + n os_n
  float *out32;                 // epi 0, 1
  double *out64;                // epi 2
  const float *lamR, *lamN;     // epi 1: divided by lamR[r] + lamN[n] - sigma
  float sigma;
  const double *sigma_dev;      // nullable: the shift read on the device (takes precedence)
  int epi;                      // 0 FP32 store, 1 FP32 store after the division, 2 FP64 store
  int *err;                     // nonzero after a timed-out wait
};

// Instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1), A and B TF32 (bits
// 7-9 and 10-12 = 2), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32_f32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(tc::smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(tc::smem_addr(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns (thread `lane` gets its lane's 32 values)
__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// One CTA computes the 128 x BN tile (m0, n0) of C = A B^T.  Warp 0 lane 0 loads (TMA),
// warp 1 lane 0 issues the MMAs, warp 2 owns the tensor memory, all four warps run the
// epilogue (warp w reads TMEM lanes 32 w .. 32 w + 31, one accumulator row per thread).
// Launched as a dependent of the previous pass: the set-up and the loads of the B operand
// (the constant eigenbases) run before pdl_wait, the A operand (the previous pass's
// output) is loaded and the output written after it.
template <class Cfg>
__device__ __forceinline__ double out_f64(float v) {
  if constexpr (Cfg::kIntCvt)
    return f64_of_f32(v);
  else
    return (double)v;
}

template <class Cfg>
__global__ void __launch_bounds__(kThreads, Cfg::kMinBlocks)
k_tf32_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            const TfArgs g) {
  constexpr int kStages = Cfg::kStages;
  constexpr uint32_t kBTileMax = Cfg::kBTile;
  extern __shared__ uint8_t smem_raw[];
  __shared__ int abort_flag;
  uint8_t *base = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int BN = g.BN;
  const uint32_t btile = (uint32_t)BN * kBK * 4;
  uint8_t *sA = base;
  uint8_t *sB = base + kStages * kATile;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sB + kStages * kBTileMax);
  uint64_t *full = bars, *empty = bars + kStages, *accum = bars + 2 * kStages;
  uint32_t *holder = reinterpret_cast<uint32_t *>(accum + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int KB = (g.K + kBK - 1) / kBK;

  if (threadIdx.x == 0) {
    pdl_trigger();
    for (int i = 0; i < kStages; ++i) {
      tc::mbar_init(&full[i], 1);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(accum, 1);
    abort_flag = 0;
    tc::fence_barrier_init();
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
  }
  if (warp == 2) tc::tmem_alloc(holder, Cfg::kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *holder;

  if (warp == 0 && lane == 0) {
    // ---- producer: the first stages' B tiles before the wait for the previous pass
    int last[kStages];
    for (int i = 0; i < kStages; ++i) last[i] = -1;
    const int pre = KB < kStages ? KB : kStages;
    for (int kb = 0; kb < pre; ++kb) {
      tc::mbar_arrive_expect_tx(&full[kb], kATile + btile);
      tma_load_2d(sB + kb * kBTileMax, &tmB, &full[kb], kb * kBK, n0);
      last[kb] = 0;
    }
    pdl_wait();
    for (int kb = 0; kb < pre; ++kb) tma_load_2d(sA + kb * kATile, &tmA, &full[kb], kb * kBK, m0);
    bool ok = true;
    for (int kb = pre; kb < KB; ++kb) {
      const int s = kb % kStages;
      const uint32_t ph = (uint32_t)(kb / kStages);
      if (!tc::mbar_wait(&empty[s], (ph & 1u) ^ 1u, g.err, 11)) {
        ok = false;
        break;
      }
      tc::mbar_arrive_expect_tx(&full[s], kATile + btile);
      tma_load_2d(sA + s * kATile, &tmA, &full[s], kb * kBK, m0);
      tma_load_2d(sB + s * kBTileMax, &tmB, &full[s], kb * kBK, n0);
      last[s] = (int)(ph & 1u);
    }
    if (!ok) {
      // wind down: let every copy this thread started land before the CTA exits
      atomicExch(&abort_flag, 1);
      for (int i = 0; i < kStages; ++i)
        if (last[i] >= 0) tc::mbar_wait(&full[i], (uint32_t)last[i], nullptr, 0);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: 4 MMAs of K = 8 per 32-wide K block
    const uint32_t idesc = idesc_tf32_f32(kBM, BN);
    bool ok = true;
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % kStages;
      const uint32_t ph = (uint32_t)(kb / kStages);
      if (!tc::mbar_wait(&full[s], ph & 1u, g.err, 12)) {
        ok = false;
        break;
      }
      tc::tc_fence_after();
      const uint32_t abase = tc::smem_addr(sA + s * kATile);
      const uint32_t bbase = tc::smem_addr(sB + s * kBTileMax);
#pragma unroll
      for (int kk = 0; kk < kBK / 8; ++kk)
        mma_tf32(tmem, tc::smem_desc_sw128(abase + kk * 32), tc::smem_desc_sw128(bbase + kk * 32),
                 idesc, (kb == 0 && kk == 0) ? 0u : 1u);
      tc::mma_commit(&empty[s]);  // the stage is free once these MMAs are done
    }
    if (!ok) atomicExch(&abort_flag, 1);
    // signal the epilogue (after a failure: only so that nothing is in flight at exit)
    tc::mma_commit(accum);
  }
  __syncwarp();

  // ---- epilogue (its stores follow the previous pass's completion: pdl_wait)
  pdl_wait();
  bool ok = tc::mbar_wait(accum, 0, g.err, 13);
  ok = __all_sync(0xffffffffu, ok);
  const int aborted = __shfl_sync(0xffffffffu, *((volatile int *)&abort_flag), 0);
  tc::tc_fence_after();
  if (ok && !aborted && KB > 0) {
    const int m = m0 + 32 * warp + lane;
    const bool mvalid = m < g.M;
    const int v = mvalid ? m / g.R : 0;
    const int r = m - v * g.R;
    const long long rowoff = (long long)v * g.os_v + (long long)r * g.os_r;
    const float sig = g.sigma_dev ? (float)*g.sigma_dev : g.sigma;
    const float lr = (g.epi == 1 && mvalid) ? g.lamR[r] - sig : 0.f;
    const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
    // contiguous rows (os_n = 1) are written 16 bytes at a time when aligned
    const bool vec =
        g.os_n == 1 && ((g.epi == 2) ? ((rowoff & 1) == 0 &&
                                        (reinterpret_cast<uintptr_t>(g.out64) & 15) == 0)
                                     : ((rowoff & 3) == 0 &&
                                        (reinterpret_cast<uintptr_t>(g.out32) & 15) == 0));
    for (int c = 0; c < BN; c += 32) {
      uint32_t d[32];
      tmem_ld_x32(trow + (uint32_t)c, d);
      tc::tmem_ld_wait();
      if (!mvalid) continue;
      const int nb = n0 + c;
      const int lim = BN - c < 32 ? BN - c : 32;  // the last chunk may end inside the tile
      float val[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        val[q] = __uint_as_float(d[q]);
        if (g.epi == 1) val[q] = __fdividef(val[q], (nb + q < g.N ? g.lamN[nb + q] : 1.f) + lr);
      }
      if (vec && lim == 32 && nb + 32 <= g.N) {
        if (g.epi == 2) {
          double2 *o = reinterpret_cast<double2 *>(g.out64 + rowoff + nb);
#pragma unroll
          for (int q = 0; q < 16; ++q) o[q] = make_double2(out_f64<Cfg>(val[2 * q]), out_f64<Cfg>(val[2 * q + 1]));
        } else {
          float4 *o = reinterpret_cast<float4 *>(g.out32 + rowoff + nb);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            o[q] = make_float4(val[4 * q], val[4 * q + 1], val[4 * q + 2], val[4 * q + 3]);
        }
      } else {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int n = nb + q;
          if (q >= lim || n >= g.N) break;
          const long long idx = rowoff + (long long)n * g.os_n;
          if (g.epi == 2)
            g.out64[idx] = out_f64<Cfg>(val[q]);
          else
            g.out32[idx] = val[q];
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 2) tc::tmem_dealloc(tmem, Cfg::kTmemCols);
}

// FP64 [rows][cols] -> FP32 [rows][ld] (ld >= cols; padding left as is): block b takes rows
// b, b + grid, ...; a thread converts 2 consecutive values of a row per step.
__global__ void k_to_f32_rows(const double *__restrict__ x, float *__restrict__ y, long long rows,
                              int cols, int ld) {
  if (threadIdx.x == 0) pdl_trigger();  // pass 1 may be scheduled (it waits for this grid)
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const double *xr = x + r * cols;
    float *yr = y + r * ld;
    for (int c = 2 * threadIdx.x; c < cols; c += 2 * blockDim.x) {
      if (c + 1 < cols) {
        yr[c] = (float)xr[c];
        yr[c + 1] = (float)xr[c + 1];
      } else {
        yr[c] = (float)xr[c];
      }
    }
  }
}

// y[i] = x[i], FP64 -> FP32, i < n (contiguous rows, ld = cols), grid-strided: two values
// per thread and step when x and y are 16- and 8-byte aligned (VEC), else one
template <bool VEC>
__global__ void k_to_f32_flat(const double *__restrict__ x, float *__restrict__ y, long long n) {
  if (threadIdx.x == 0) pdl_trigger();  // pass 1 may be scheduled (it waits for this grid)
  if (!VEC) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
      y[i] = f32_of_f64(x[i]);
    return;
  }
  const long long n2 = n >> 1;
  const double2 *x2 = reinterpret_cast<const double2 *>(x);
  float2 *y2 = reinterpret_cast<float2 *>(y);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n2;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = x2[i];
    y2[i] = make_float2(f32_of_f64(v.x), f32_of_f64(v.y));
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) y[n - 1] = f32_of_f64(x[n - 1]);
}

// dst[r][c] = src[r][c] (or src[c][r] when transposed), rows x cols, ld padded, FP32
__global__ void k_pad_copy(const float *__restrict__ src, int rows, int cols, int transpose,
                           float *__restrict__ dst, int ld) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * ld; e += gridDim.x * blockDim.x) {
    const int r = e / ld, c = e - (e / ld) * ld;
    dst[e] = c < cols ? (transpose ? src[(long long)c * rows + r] : src[(long long)r * cols + c]) : 0.f;
  }
}

// out[(i1 n2 + i2) n3 + i3] = l1[i1] + l2[i2] + l3[i3]: the eigenvalue sums of three modes
// over the rows of the 2D preconditioner's dividing pass
__global__ void k_lam_sum3(const float *__restrict__ l1, const float *__restrict__ l2,
                           const float *__restrict__ l3, int n1, int n2, int n3,
                           float *__restrict__ out) {
  const long long total = (long long)n1 * n2 * n3;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i3 = (int)(e % n3);
    const long long r = e / n3;
    out[e] = l1[r / n2] + l2[r % n2] + l3[i3];
  }
}

// ------------------------------------ host ------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// Tensor map over an FP32 matrix [rows][ld], K = cols contiguous: boxes of 32 K x box_rows
// rows, 128-byte swizzle, zero fill outside cols x rows.
bool make_f32_map(CUtensorMap *map, const float *base, int cols, long long rows, int ld,
                  int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (ld * 4) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || cols > ld)
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int pad4(int n) { return (n + 3) & ~3; }

// tile width for N columns: as few tiles of at most 256 as possible, each a multiple of 16
// Output tile width for N columns when the M side has mtiles tiles: the fewest tiles of at
// most kBNMax columns, then more (narrower, down to about 64 columns) tiles while all of
// them fit in one wave on the 152 SMs.  The passes are latency-bound (a short K loop per
// CTA), so spreading a pass over more SMs shortens it; below 64 columns an MMA costs as
// much as at 64 (about 45 issue cycles), so narrower tiles would only add MMAs.
int tile_n(int N, int mtiles) {
  int tiles = (N + kBNMax - 1) / kBNMax;
  while (tiles + 1 <= (N + 63) / 64 && (long long)(tiles + 1) * mtiles <= 152) ++tiles;
  const int bn = (N + tiles - 1) / tiles;
  return (bn + 15) & ~15;
}

template <class Cfg>
void launch_tf32_gemm(const CUtensorMap &ta, const CUtensorMap &tb, const TfArgs &g,
                      cudaStream_t s) {
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(k_tf32_gemm<Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)Cfg::kSmem);
  });
  count_launch();
  launch_pdl(k_tf32_gemm<Cfg>,
             dim3((unsigned)((g.M + kBM - 1) / kBM), (unsigned)((g.N + g.BN - 1) / g.BN)),
             dim3(kThreads), Cfg::kSmem, s, ta, tb, g);
}

}  // namespace

// Padded FP32 eigenbases and the tensor maps of the four passes: the operator maps are
// built once; the workspace maps cover whole buffers (rows beyond a call's M are read
// but their results are not stored) and are rebuilt only when the workspace changes.
struct TfOperator {
  int nx = 0, ny = 0, XP = 0, YP = 0, BNx = 0, BNy = 0;
  float *Sx = nullptr, *STx = nullptr, *Sy = nullptr, *STy = nullptr;  // padded copies
  int *err = nullptr;  // device flag of timed-out waits
  CUtensorMap mSTy, mSTx, mSx, mSy;  // B operands of passes 1 .. 4
  const void *ws0 = nullptr, *ws1 = nullptr;
  long long wscap = -1;
  CUtensorMap mA[4];                 // A operands of passes 1 .. 4
  // 2D: per mode k the tile width and the B operands S_k^T (forward) and S_k (backward)
  // over the FP32 eigenbases themselves (n_k is a multiple of 4, so rows need no padding);
  // mA4[k] the input of the passes that contract mode k; lamR the sums of the eigenvalues
  // of modes 1, 2, 3 over the rows of the dividing pass
  bool two_d = false;
  int n4[4] = {0, 0, 0, 0}, BN4[4] = {0, 0, 0, 0};
  float *lamR = nullptr;
  CUtensorMap mST4[4], mS4[4], mA4[4];
};

void free_tf_operator(TfOperator *t) {
  if (!t) return;
  cudaFree(t->Sx);
  cudaFree(t->lamR);
  cudaFree(t->err);
  delete t;
}

bool tf_prec_supported(const DevOperator &op) {
  if (op.nmodes == 2) return true;
  if (op.nmodes != 4) return false;
  for (int k = 0; k < 4; ++k)
    if (op.n[k] < 4 || op.n[k] > 128 || op.n[k] % 4 != 0) return false;
  return true;
}

// 2D: every mode 4 .. 128 points, a multiple of 4 (TMA rows of 16 bytes)
int ensure_tf_operator_2d(const DevOperator &op) {
  TfOperator *t = new TfOperator();
  t->two_d = true;
  bool ok = true;
  for (int k = 0; k < 4; ++k) {
    const int n = op.n[k];
    if (n < 4 || n > 128 || n % 4 != 0) {
      delete t;
      return TPS_ERR_INVALID_ARG;
    }
    t->n4[k] = n;
    const int tiles = (n + Cfg2::kBNMax - 1) / Cfg2::kBNMax;
    t->BN4[k] = (((n + tiles - 1) / tiles) + 15) & ~15;
    ok = ok && make_f32_map(&t->mST4[k], op.STf[k], n, n, n, t->BN4[k]) &&
         make_f32_map(&t->mS4[k], op.Sf[k], n, n, n, t->BN4[k]);
  }
  const long long nr = (long long)op.n[1] * op.n[2] * op.n[3];
  if (!ok || cudaMalloc((void **)&t->lamR, nr * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void **)&t->err, sizeof(int)) != cudaSuccess ||
      cudaMemset(t->err, 0, sizeof(int)) != cudaSuccess) {
    free_tf_operator(t);
    return ok ? TPS_ERR_NOMEM : TPS_ERR_INVALID_ARG;
  }
  k_lam_sum3<<<256, 256>>>(op.lamf[1], op.lamf[2], op.lamf[3], op.n[1], op.n[2], op.n[3],
                           t->lamR);
  if (cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    free_tf_operator(t);
    return TPS_ERR_CUDA;
  }
  op.tf = t;
  return TPS_OK;
}

int ensure_tf_operator(const DevOperator &op) {
  if (op.tf) return TPS_OK;
  if (op.nmodes == 4) return ensure_tf_operator_2d(op);
  if (op.nmodes != 2) return TPS_ERR_INVALID_ARG;
  TfOperator *t = new TfOperator();
  t->nx = op.n[0];
  t->ny = op.n[1];
  t->XP = pad4(t->nx);
  t->YP = pad4(t->ny);
  // tiles sized for blocks of 8 vectors (the solver's usual block); other counts work too
  t->BNx = tile_n(t->nx, (8 * t->ny + kBM - 1) / kBM);
  t->BNy = tile_n(t->ny, (8 * t->nx + kBM - 1) / kBM);
  const size_t fx = (size_t)t->nx * t->XP, fy = (size_t)t->ny * t->YP;
  if (cudaMalloc((void **)&t->Sx, (2 * fx + 2 * fy) * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void **)&t->err, sizeof(int)) != cudaSuccess ||
      cudaMemset(t->err, 0, sizeof(int)) != cudaSuccess) {
    free_tf_operator(t);
    return TPS_ERR_NOMEM;
  }
  t->STx = t->Sx + fx;
  t->Sy = t->STx + fx;
  t->STy = t->Sy + fy;
  // Sf[k] is S_k row-major (S[i][j]); the transposes are read from it transposed
  k_pad_copy<<<256, 256>>>(op.Sf[0], t->nx, t->nx, 0, t->Sx, t->XP);
  k_pad_copy<<<256, 256>>>(op.Sf[0], t->nx, t->nx, 1, t->STx, t->XP);
  k_pad_copy<<<256, 256>>>(op.Sf[1], t->ny, t->ny, 0, t->Sy, t->YP);
  k_pad_copy<<<256, 256>>>(op.Sf[1], t->ny, t->ny, 1, t->STy, t->YP);
  const bool maps = make_f32_map(&t->mSTy, t->STy, t->ny, t->ny, t->YP, t->BNy) &&
                    make_f32_map(&t->mSTx, t->STx, t->nx, t->nx, t->XP, t->BNx) &&
                    make_f32_map(&t->mSx, t->Sx, t->nx, t->nx, t->XP, t->BNx) &&
                    make_f32_map(&t->mSy, t->Sy, t->ny, t->ny, t->YP, t->BNy);
  if (!maps || cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess ||
      cudaGetLastError() != cudaSuccess) {
    free_tf_operator(t);
    return maps ? TPS_ERR_CUDA : TPS_ERR_INVALID_ARG;
  }
  op.tf = t;
  return TPS_OK;
}

long long tf_prec_workspace_floats(const DevOperator &op, int nvec) {
  if (op.nmodes == 4) return (long long)nvec * op.N;
  const long long a = (long long)nvec * op.n[0] * pad4(op.n[1]);
  const long long b = (long long)nvec * op.n[1] * pad4(op.n[0]);
  return a > b ? a : b;
}

// 2D (four modes a, b, c, d = x1, x2, y1, y2; C order, d fastest): eight passes, each
// contracting the last index of its input and storing its output index first, so the
// indices rotate by one per pass and every pass reads its contraction index contiguously:
//   X[a][b][c][d] -> T1[j_d][a][b][c] -> T2[j_c][j_d][a][b] -> T3[j_b][j_c][j_d][a]
//   -> T4[j_a][j_b][j_c][j_d] divided by lambda_a + lambda_b + lambda_c + lambda_d - sigma
// (B = S_k^T: t_j = sum_i x_i S_k[i][j]), then the same four contractions with B = S_k
// (u_i = sum_j t_j S_k[i][j]), the last one storing FP64 in the original order.  A pass over
// mode k is C = A B^T with A = nvec N / n_k rows of n_k values; its output element (v, row r,
// column n) lies at v N + n (N / n_k) + r.
int launch_apply_prec_tf32_2d(const DevOperator &op, const double *r, double *out, int nvec,
                              double sigma, ApplyWorkspace &ws, cudaStream_t s,
                              const double *sigma_dev) {
  TfOperator *t = op.tf;
  if (tf_prec_workspace_floats(op, nvec) > 2 * ws.capacity) return TPS_ERR_INVALID_ARG;
  const long long N = op.N;
  float *bufA = reinterpret_cast<float *>(ws.t0), *bufB = reinterpret_cast<float *>(ws.t1);
  // the passes over modes 3 and 1 read bufA, those over modes 2 and 0 read bufB
  auto inbuf = [&](int k) { return (k & 1) ? bufA : bufB; };
  if (t->ws0 != ws.t0 || t->ws1 != ws.t1 || t->wscap != ws.capacity) {
    const long long fl = 2 * ws.capacity;  // floats per buffer
    for (int k = 0; k < 4; ++k)
      if (!make_f32_map(&t->mA4[k], inbuf(k), t->n4[k], fl / t->n4[k], t->n4[k], kBM))
        return TPS_ERR_INVALID_ARG;
    t->ws0 = ws.t0;
    t->ws1 = ws.t1;
    t->wscap = ws.capacity;
  }
  {
    // the rows (n_3 values, a multiple of 4) need no padding: one flat conversion
    const long long n = (long long)nvec * N;
    long long blocks = (n / 2 + 255) / 256;
    if (blocks > 152LL * 8) blocks = 152LL * 8;
    count_launch();
    if ((reinterpret_cast<uintptr_t>(r) & 15) == 0 && (reinterpret_cast<uintptr_t>(bufA) & 7) == 0)
      k_to_f32_flat<true><<<(unsigned)blocks, 256, 0, s>>>(r, bufA, n);
    else
      k_to_f32_flat<false><<<(unsigned)blocks, 256, 0, s>>>(r, bufA, n);
  }
  TfArgs g{};
  g.err = t->err;
  g.sigma = (float)sigma;
  g.sigma_dev = sigma_dev;
  g.os_v = N;
  g.os_r = 1;
  for (int pass = 0; pass < 8; ++pass) {
    const int k = 3 - (pass & 3);
    const int n = t->n4[k];
    g.M = (int)((long long)nvec * (N / n));
    g.N = n;
    g.K = n;
    g.R = (int)(N / n);
    g.BN = t->BN4[k];
    g.os_n = N / n;
    g.epi = pass == 3 ? 1 : (pass == 7 ? 2 : 0);
    g.out32 = (k & 1) ? bufB : bufA;  // the next pass's input
    g.out64 = out;
    g.lamR = t->lamR;
    g.lamN = op.lamf[0];
    launch_tf32_gemm<Cfg2>(t->mA4[k], pass < 4 ? t->mST4[k] : t->mS4[k], g, s);
  }
  return TPS_OK;
}

int launch_apply_prec_tf32(const DevOperator &op, const double *r, double *out, int nvec,
                           double sigma, ApplyWorkspace &ws, cudaStream_t s,
                           const double *sigma_dev) {
  if (nvec <= 0) return TPS_OK;
  TfOperator *t = op.tf;
  if (t && t->two_d && op.nmodes == 4)
    return launch_apply_prec_tf32_2d(op, r, out, nvec, sigma, ws, s, sigma_dev);
  if (!t || op.nmodes != 2) return TPS_ERR_INVALID_ARG;
  if (tf_prec_workspace_floats(op, nvec) > 2 * ws.capacity) return TPS_ERR_INVALID_ARG;
  const int nx = t->nx, ny = t->ny, XP = t->XP, YP = t->YP;
  float *bufA = reinterpret_cast<float *>(ws.t0), *bufB = reinterpret_cast<float *>(ws.t1);
  if (t->ws0 != ws.t0 || t->ws1 != ws.t1 || t->wscap != ws.capacity) {
    const long long fl = 2 * ws.capacity;  // floats per buffer
    if (!make_f32_map(&t->mA[0], bufA, ny, fl / YP, YP, kBM) ||
        !make_f32_map(&t->mA[1], bufB, nx, fl / XP, XP, kBM) ||
        !make_f32_map(&t->mA[2], bufA, nx, fl / XP, XP, kBM) ||
        !make_f32_map(&t->mA[3], bufB, ny, fl / YP, YP, kBM))
      return TPS_ERR_INVALID_ARG;
    t->ws0 = ws.t0;
    t->ws1 = ws.t1;
    t->wscap = ws.capacity;
  }
  {
    long long blocks = (long long)nvec * nx;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    count_launch();
    k_to_f32_rows<<<(unsigned)blocks, 128, 0, s>>>(r, bufA, (long long)nvec * nx, ny, YP);
  }
  TfArgs g{};
  g.err = t->err;
  g.sigma = (float)sigma;
  g.sigma_dev = sigma_dev;
  // pass 1: t0T[v][j][x] = sum_y r[v][x][y] S_y[y][j]
  g.M = nvec * nx; g.N = ny; g.K = ny; g.R = nx; g.BN = t->BNy;
  g.os_v = (long long)ny * XP; g.os_r = 1; g.os_n = XP;
  g.out32 = bufB; g.epi = 0;
  launch_tf32_gemm<Cfg1>(t->mA[0], t->mSTy, g, s);
  // pass 2: t1T[v][j][i] = sum_x t0T[v][j][x] S_x[x][i] / (lambda_x[i] + lambda_y[j] - sigma)
  g.M = nvec * ny; g.N = nx; g.K = nx; g.R = ny; g.BN = t->BNx;
  g.os_v = (long long)ny * XP; g.os_r = XP; g.os_n = 1;
  g.out32 = bufA; g.epi = 1; g.lamR = op.lamf[1]; g.lamN = op.lamf[0];
  launch_tf32_gemm<Cfg1>(t->mA[1], t->mSTx, g, s);
  // pass 3: t2[v][x][j] = sum_i S_x[x][i] t1T[v][j][i]
  g.M = nvec * ny; g.N = nx; g.K = nx; g.R = ny; g.BN = t->BNx;
  g.os_v = (long long)nx * YP; g.os_r = 1; g.os_n = YP;
  g.out32 = bufB; g.epi = 0;
  launch_tf32_gemm<Cfg1>(t->mA[2], t->mSx, g, s);
  // pass 4: out[v][x][y] = sum_j t2[v][x][j] S_y[y][j]
  g.M = nvec * nx; g.N = ny; g.K = ny; g.R = nx; g.BN = t->BNy;
  g.os_v = (long long)nx * ny; g.os_r = ny; g.os_n = 1;
  g.out64 = out; g.epi = 2;
  launch_tf32_gemm<Cfg1>(t->mA[3], t->mSy, g, s);
  return TPS_OK;
}

// Reads (synchronously) and clears the operator's timed-out-wait flag.
int tf_operator_status(const DevOperator &op) {
  if (!op.tf) return 0;
  int h = 0;
  if (cudaMemcpy(&h, op.tf->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  if (h && (cudaMemset(op.tf->err, 0, sizeof(int)) != cudaSuccess ||
            cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess))
    return -1;
  return h;
}

}  // namespace tps
