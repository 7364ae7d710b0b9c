// FP64-accurate tall-skinny block updates C = beta C + alpha A Y on the tensor cores
// (the Ritz vectors X = V Y and HX = (HV) Y, restarts, and the projections of the
// orthogonalisation in Sec. 4.1).  A is n x p (p <= 64 per call, column-major, n up to
// millions), Y is p x q with q <= 8 per CTA group.
//
// The products are emulated by error-free digit splitting (the Ozaki scheme: Ozaki,
// Ogita, Oishi & Rump, Numer. Algorithms 59, 2012), as in the H-apply:
//  * row r of A gets the exponent E_r with |A[r][k]| < 2^E_r for all k, column j of
//    alpha Y the exponent F_j; each value becomes the integer round(x 2^(54 - E)) and is
//    written in nine balanced base-64 digits, most significant first, |d| <= 64;
//  * the digit pairs (i, j) with i + j <= 9 are multiplied in BF16 (small integers are
//    exact) and the pairs of one level l = i + j are summed in one FP32 accumulator:
//    every partial sum is an integer below 64 (l + 1) 2^12 < 2^24 (p <= 64), hence exact;
//  * the levels are combined in two int64 Horner sums and scaled by 2^(E_r + F_j).
// The result has the row-wise accuracy of the FP64 product (2^-55 of the row maximum of
// A times sum_k |alpha Y[k][j]|, plus the truncation of the levels l > 9 below that).
//
// The MMA is the warp-level mma.sync m16n8k16 (BF16 in, FP32 out): the output is only
// q <= 8 columns wide, and a tcgen05.mma costs its issuing thread about 45 cycles
// whatever N (measured: 367 FLOP/clk/SM at M = 64, N = 8), while mma.sync m16n8k16 runs at
// 2 cycles per warp instruction per SM (2046 FLOP/clk/SM).  The 53 digit products per
// multiply-add then cost less than the one FP64 FMA they replace on GB300's FP64 pipe
// (4 FLOP/clk/SM).  The digit splitting of A runs on the FP32 pipe: the 54-bit integer
// is cut into three 18-bit chunks, each exact in FP32, and each chunk into three digits
// by two roundings.
#include <cuda_bf16.h>

#include "tps_internal.h"

namespace tps {
namespace {

constexpr int kUT = 128;   // threads per CTA: 4 warps, each 16 rows at a time
constexpr int kUS = 9;     // digits per operand
constexpr int kUL = 10;    // levels kept: i + j <= 9
constexpr int kUKT = 4;    // k tiles of 16 (p <= 64)

__device__ __forceinline__ unsigned raw_exp(double x) {
  return (unsigned)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// round(x 2^(54 - E)), E = raw_max - 1022 (so |x| < 2^E), by integer arithmetic on the
// FP64 fields; subnormals flush to zero.  |result| <= 2^54.
__device__ __forceinline__ long long scaled54(double x, unsigned raw_max) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((u >> 52) & 0x7FF);
  if (ex == 0 || raw_max == 0) return 0;
  const long long mant = (long long)((u & ((1ULL << 52) - 1)) | (1ULL << 52));
  const int sh = ex - 1075 + 54 - ((int)raw_max - 1022);
  long long q;
  if (sh >= 0)
    q = mant << sh;
  else if (sh > -63)
    q = (mant + (1LL << (-sh - 1))) >> (-sh);
  else
    q = 0;
  return (u >> 63) ? -q : q;
}

// The nine digits of x: x 2^(54 - E) = sum_i d[i] 64^(8 - i), |d[i]| <= 64.
__device__ __forceinline__ void digits9(double x, unsigned raw_max, float (&d)[kUS]) {
  const long long q = scaled54(x, raw_max);
  const float sg = q < 0 ? -1.f : 1.f;
  const unsigned long long a = (unsigned long long)(q < 0 ? -q : q);
  const unsigned ch[3] = {(unsigned)(a >> 36), (unsigned)((a >> 18) & 0x3FFFFu),
                          (unsigned)(a & 0x3FFFFu)};
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    float f = (float)ch[t];                        // <= 2^18: exact
    const float d0 = rintf(f * (1.f / 4096.f));    // 0 .. 64
    f = fmaf(-d0, 4096.f, f);                      // |f| <= 2048
    const float d1 = rintf(f * (1.f / 64.f));      // |d1| <= 32
    f = fmaf(-d1, 64.f, f);                        // |f| <= 32
    d[3 * t] = sg * d0;
    d[3 * t + 1] = sg * d1;
    d[3 * t + 2] = sg * f;
  }
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x in the low half
  return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void mma_16816(float (&c)[4], const uint32_t (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

__device__ __forceinline__ double pow2d(int e) {
  e = e < -1022 ? -1022 : (e > 1023 ? 1023 : e);
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// CTA (x, s, z): columns j0 = 8 z .. j0 + 7 of batch item s, row blocks of 64 (16 per
// warp) strided over gridDim.x.  Fragment layout of m16n8k16 (g = lane / 4, c = lane % 4):
// A regs {row g, k 2c..2c+1}, {row g+8, k 2c..}, {row g, k 2c+8..}, {row g+8, k 2c+8..};
// B regs {k 2c..2c+1, col g}, {k 2c+8.., col g}; C {row g, col 2c, 2c+1}, {row g+8, ..}.
__global__ void __launch_bounds__(kUT)
k_update_split(const double *__restrict__ A, long long lda, long long bsa, int p,
               const double *__restrict__ Y, int ldy, long long bsy, int q, double alpha,
               double beta, double *__restrict__ C, long long ldc, long long bsc,
               long long nrows, const int *__restrict__ need) {
  if (need && *need == 0) return;  // conditional product (decided on the device)
  __shared__ uint2 Bd[kUS][kUKT][32];
  __shared__ unsigned Fraw[8];
  const int s = blockIdx.y, j0 = blockIdx.z * 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, c = lane & 3;
  const int KT = (p + 15) >> 4;
  const double *Ys = Y + s * bsy;
  // column exponents of alpha Y (8 columns, p <= 64 rows): 16 threads per column, each
  // over every 16th row, then a max across the 16 lanes
  {
    const int jl = threadIdx.x >> 4, k0 = threadIdx.x & 15, j = j0 + jl;
    unsigned m = 0;
    if (j < q)
#pragma unroll
      for (int k = k0; k < 64; k += 16)
        if (k < p) m = max(m, raw_exp(alpha * Ys[(long long)j * ldy + k]));
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (k0 == 0) Fraw[jl] = m;
  }
  __syncthreads();
  // B fragments of the nine digit planes of alpha Y: thread (kt, lane) packs its own
  {
    const int kt = threadIdx.x >> 5;
    if (kt < kUKT) {
      const int j = j0 + g;
      float dv[4][kUS];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = 16 * kt + 2 * c + (e & 1) + 8 * (e >> 1);
        const double y = (j < q && k < p) ? alpha * Ys[(long long)j * ldy + k] : 0.0;
        digits9(y, Fraw[g], dv[e]);
      }
#pragma unroll
      for (int i = 0; i < kUS; ++i)
        Bd[i][kt][lane] = make_uint2(pack_bf16(dv[0][i], dv[1][i]), pack_bf16(dv[2][i], dv[3][i]));
    }
  }
  __syncthreads();
  const double *As = A + s * bsa;
  double *Cs = C + s * bsc;
  const long long nblk = (nrows + 15) >> 4;
  for (long long blk = (long long)blockIdx.x * 4 + warp; blk < nblk; blk += (long long)gridDim.x * 4) {
    const long long ra = blk * 16 + g, rb = ra + 8;
    const bool va = ra < nrows, vb = rb < nrows;
    {
      // the warp's next 16-row block into L1 while this one is split and multiplied (the
      // kernel is bound by load latency): rows r and r + 8 share a 128-byte line
      const long long nr = ra + (long long)gridDim.x * 64;
      if (nr < nrows)
        for (int kt = 0; kt < KT; ++kt)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int k = 16 * kt + 2 * c + (e & 1) + 8 * (e >> 1);
            if (k < p)
              asm volatile("prefetch.global.L1 [%0];" ::"l"(As + (long long)k * lda + nr));
          }
    }
    // row exponents: the thread's k values of rows ra and rb, then across the quad
    unsigned ea = 0, eb = 0;
    for (int kt = 0; kt < KT; ++kt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = 16 * kt + 2 * c + (e & 1) + 8 * (e >> 1);
        if (k < p) {
          if (va) ea = max(ea, raw_exp(As[(long long)k * lda + ra]));
          if (vb) eb = max(eb, raw_exp(As[(long long)k * lda + rb]));
        }
      }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
      ea = max(ea, __shfl_xor_sync(0xffffffffu, ea, o));
      eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, o));
    }
    float acc[kUL][4];
#pragma unroll
    for (int l = 0; l < kUL; ++l)
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[l][t] = 0.f;
    for (int kt = 0; kt < KT; ++kt) {
      // A digit fragments: value e of register r is (row ra|rb, k 16kt + 2c + e + 8 (r>>1))
      uint32_t af[kUS][4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const bool v = (r & 1) ? vb : va;
        const long long row = (r & 1) ? rb : ra;
        const unsigned er = (r & 1) ? eb : ea;
        float d0[kUS], d1[kUS];
        const int k = 16 * kt + 2 * c + 8 * (r >> 1);
        digits9((v && k < p) ? As[(long long)k * lda + row] : 0.0, er, d0);
        digits9((v && k + 1 < p) ? As[(long long)(k + 1) * lda + row] : 0.0, er, d1);
#pragma unroll
        for (int i = 0; i < kUS; ++i) af[i][r] = pack_bf16(d0[i], d1[i]);
      }
#pragma unroll
      for (int j = 0; j < kUS; ++j) {
        const uint2 b = Bd[j][kt][lane];
#pragma unroll
        for (int i = 0; i < kUS; ++i)
          if (i + j < kUL) mma_16816(acc[i + j], af[i], b);
      }
    }
    // combine the levels: sum_l D_l 2^(-6 (l + 2)), hi = levels 0..4, lo = levels 5..9
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const bool v = (t & 2) ? vb : va;
      const int jl = 2 * c + (t & 1);
      const int j = j0 + jl;
      if (!v || j >= q) continue;
      long long hi = 0, lo = 0;
#pragma unroll
      for (int l = 0; l < kUL; ++l) {
        const long long dl = (long long)__float2int_rn(acc[l][t]);
        if (l < kUL / 2)
          hi = hi * 64 + dl;
        else
          lo = lo * 64 + dl;
      }
      const unsigned er = (t & 2) ? eb : ea, fr = Fraw[jl];
      double val = 0.0;
      if (er && fr) {
        const int E = (int)er - 1022 + (int)fr - 1022;
        val = fma((double)lo, pow2d(E - 6 * (kUL + 1)), (double)hi * pow2d(E - 6 * (kUL / 2 + 1)));
      }
      double *dst = Cs + (long long)j * ldc + ((t & 2) ? rb : ra);
      *dst = (beta == 0.0) ? val : fma(beta, *dst, val);
    }
  }
}

}  // namespace

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
  const long long blocks64 = (nrows + 63) / 64;
  // p is processed in slabs of 64 rows of Y; the first slab applies beta
  for (int i0 = 0; i0 < p; i0 += 64) {
    const int pp = p - i0 < 64 ? p - i0 : 64;
    const long long gx = blocks64 < 152LL * 8 ? blocks64 : 152LL * 8;
    const dim3 grid((unsigned)gx, batch, (q + 7) / 8);
    count_launch();
    k_update_split<<<grid, kUT, 0, s>>>(A + (long long)i0 * lda, lda, bsa, pp, Y + i0, ldy, bsy, q,
                                        alpha, i0 == 0 ? beta : 1.0, C, ldc, bsc, nrows, need);
  }
}

}  // namespace tps
