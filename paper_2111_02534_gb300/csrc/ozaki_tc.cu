// FP64-accurate mode products on the tcgen05 tensor cores (1D H-apply, Eq. tensor_op1D).
//
// GB300's FP64 FMA pipe peaks at 1.26 TFLOP/s while its BF16 tensor cores run three
// orders of magnitude faster, so the FP64 mode products are emulated by error-free
// splitting (the Ozaki scheme: Ozaki, Ogita, Oishi & Rump, "Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012), with BF16 digits and exact FP32
// accumulation:
//
//  * Every row r of an FP64 operand X (rows = output index, columns = contraction index)
//    gets the exponent E_r with |X[r][k]| < 2^E_r.  X[r][k] 2^(S*beta - E_r) is rounded to
//    an integer and written in S balanced base-2^beta digits d_1..d_S (beta = 6),
//    |d_1| <= 64 and |d_i| <= 32 otherwise, so
//    X[r][k] = 2^E_r sum_i d_i[r][k] 2^(-i beta) up to 2^(E_r - S beta - 1).  Small
//    integers are exact in BF16.
//  * C = A B^T is the sum over digit pairs (i, j) of 2^(E_A + E_B - (i+j) beta) times the
//    integer matrix D_ij = d_i(A) d_j(B)^T.  Pairs with i + j <= 11 (1-based) are kept.  The
//    pairs of one level l = i + j accumulate in one FP32 TMEM accumulator: every partial
//    sum is an integer of magnitude at most K 2^10 (l + 1) < 2^24 for K <= 1365, hence
//    exact.
//  * The wave function gets 9 digits (54 bits, rounding error random from element to
//    element).  The mode matrices get 10: their rows are dominated by the diagonal, so a
//    per-row scale leaves the small far-off-diagonal entries with an absolute rounding of
//    2^-55 of the diagonal, and since D2 is circulant these errors repeat in every row;
//    their row sum would act on smooth wave functions like a constant potential of
//    ~1e-13 (measured as a uniform eigenvalue shift).  The tenth digit (pairs with the
//    wave function's leading digit) puts that sum near 1e-16.
//  * The epilogue converts each level to an integer, combines the levels in two int64
//    Horner sums (exact) and forms the FP64 result with one conversion pair and one FMA.
//  * The 2D mode products contract over at most 128 points, short enough for base-256
//    digits (beta = 8, every digit in [-128, 128], still exact in BF16): seven for the
//    wave function's fibers (55 bits), eight for the mode matrices (62 bits), and the 35
//    pairs with i + j <= 8 (1-based) in eight accumulators, every partial sum below
//    7 * 2^14 * 146 < 2^24 for K <= 146 (54 pairs and ten levels in base 64).
//
// The 1D H-apply out = K_x P + P K_y^T + (V - theta) P (P = psi as n_x x n_y) runs as two
// such products in the transposed orientation (rows of C = the y index, so that one warp
// stores 32 consecutive y of an output row):
//    C1[y][x] = sum_y' K_y[y][y'] P[x][y']     A = slices of K_y,  B = slices of P
//    C2[y][x] = sum_x' P^T[y][x'] K_x[x][x']   A = slices of P^T,  B = slices of K_x
// with the potential term fused into the first epilogue; both products run in one launch
// and add their tiles to the zeroed output (two terms per element, so the FP64 atomic sum
// is order-independent).  Operand tiles reach shared memory by TMA (128-byte swizzle,
// K-major), one thread issues tcgen05.mma into tensor memory, and eight warps drain it.
//
// The 2D H-apply (Eq. tensor_op2D) runs its four mode products one after the other, each
// over the fibers of its mode (A = fiber slices, B = K_k slices), with a persistent kernel:
// one CTA per SM takes tile after tile, its producer, MMA and epilogue warps working on
// successive tiles at once (the 48-point contraction gives short MMA loops, so a CTA per
// tile spent most of its time in the epilogue with the tensor pipe idle).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <utility>

#include "ozaki_tc.cuh"
#include "pdl.cuh"
#include "split_digits.cuh"
#include "tps_internal.h"

namespace tps {

namespace {


constexpr int kBeta = 6;
constexpr int kPsiSlices = 9;  // wave-function digits: 54 bits
constexpr int kOpSlices = 10;  // mode-matrix digits: 60 bits (see below)
constexpr int kLevels = 10;    // digit-pair levels kept: i + j <= 9 (0-based)
// 2D mode products (contraction length <= 128): base-256 digits, |d| <= 128, so a level's
// partial sums stay below 7 * 2^14 * 146 < 2^24 (exact in FP32) for K <= 146
constexpr int kPsiSlices2 = 7;  // wave-function digits: 55 bits
constexpr int kOpSlices2 = 8;   // mode-matrix digits: 62 bits
constexpr int kLevels2 = 8;     // i + j <= 7
constexpr int kMaxSlices = 10;
constexpr int kBM = 128;       // output rows per CTA (TMEM lanes)
constexpr int kBN = 48;        // output columns per CTA; kLevels * kBN <= 512 TMEM columns
constexpr int kBK = 64;        // contraction depth per stage (128-byte rows)
constexpr int kAStages = 6;  // A tiles in flight: each carries ~600 cycles of MMA work
constexpr int kBStages = 2;  // a power of two (stage index by mask)
constexpr int kThreads = 256;  // 8 warps drain the accumulators (two per TMEM lane quarter)
constexpr uint32_t kATileBytes = kBM * 128;
constexpr uint32_t kTmemCols = 512;
static_assert(kLevels * kBN <= (int)kTmemCols, "levels must fit in tensor memory");
static_assert(kBN % 16 == 0 && kBN >= 16 && kBN <= 256, "N of a 128-row MMA");

__host__ __device__ constexpr uint32_t b_slice_bytes() { return kBN * 128; }

size_t oz_smem_bytes(int SB) {
  return 1024 /* alignment slack */ + (size_t)kBStages * SB * b_slice_bytes() +
         (size_t)kAStages * kATileBytes + 8 * (2 * kAStages + 2 * kBStages + 1) + 16;
}

// -------------------------------- splitting ----------------------------------
__device__ __forceinline__ unsigned raw_exponent(double x) {
  return (unsigned)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// The nine balanced base-64 digits of a scaled integer |q| <= 2^54 (most significant first),
// as BF16 bit patterns: q is cut into three balanced 18-bit chunks by integer arithmetic and
// each chunk (exact in FP32) into three digits by two FP32 roundings, d0 = rint(c 2^-12),
// d1 = rint((c - 2^12 d0) 2^-6), d2 = c - 2^12 d0 - 2^6 d1.  Digits 1..8 lie in [-32, 32],
// the top one in [-64, 64]; every one is exact in BF16 (a hardware conversion).  The digits
// sum to q with the weights 2^(6 (8 - i)) like the digit-by-digit extraction below, which
// the mode matrices' ten-digit slices use.
__device__ __forceinline__ void digits9(long long q, uint16_t (&o)[9]) {
  long long c[3];
#pragma unroll
  for (int k = 2; k > 0; --k) {  // least significant chunks first
    long long l = q & ((1LL << 18) - 1);
    if (l >= (1LL << 17)) l -= (1LL << 18);
    c[k] = l;
    q = (q - l) >> 18;
  }
  c[0] = q;  // |q| <= 2^18
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float f = (float)c[k];
    const float d0 = rintf(f * (1.f / 4096.f));
    const float r = fmaf(-d0, 4096.f, f);
    const float d1 = rintf(r * (1.f / 64.f));
    const float d2 = fmaf(-d1, 64.f, r);
    o[3 * k] = __bfloat16_as_ushort(__float2bfloat16_rn(d0));
    o[3 * k + 1] = __bfloat16_as_ushort(__float2bfloat16_rn(d1));
    o[3 * k + 2] = __bfloat16_as_ushort(__float2bfloat16_rn(d2));
  }
}

// The S balanced base-256 digits (S = 7: |q| <= 2^55; S = 8: |q| <= 2^62) of a scaled
// integer, most significant first, as BF16 bit patterns, every digit in [-128, 128]:
// q = c0 2^48 + c1 2^24 + c2 with c1, c2 balanced 24-bit chunks (integer arithmetic), each
// chunk (exact in FP32) cut into three digits by two FP32 roundings, d0 = rint(c 2^-16),
// d1 = rint((c - 2^16 d0) 2^-8), d2 = c - 2^16 d0 - 2^8 d1; c0 is one digit (|c0| <= 128)
// for S = 7, and two, e0 = rint(c0 / 256) and c0 - 256 e0, for S = 8 (|c0| <= 2^14 + 1).
// Digit i weighs 2^(8 (S - 1 - i)).
template <int S>
__device__ __forceinline__ void digits256(long long q, uint16_t (&o)[S]) {
  static_assert(S == 7 || S == 8, "seven or eight base-256 digits");
  long long c[3];
#pragma unroll
  for (int k = 2; k > 0; --k) {  // least significant chunks first
    long long l = q & ((1LL << 24) - 1);
    if (l >= (1LL << 23)) l -= (1LL << 24);
    c[k] = l;
    q = (q - l) >> 24;
  }
  c[0] = q;
  int p = 0;
  const float f0 = (float)c[0];
  if (S == 8) {
    const float e0 = rintf(f0 * (1.f / 256.f));
    o[p++] = __bfloat16_as_ushort(__float2bfloat16_rn(e0));
    o[p++] = __bfloat16_as_ushort(__float2bfloat16_rn(fmaf(-e0, 256.f, f0)));
  } else {
    o[p++] = __bfloat16_as_ushort(__float2bfloat16_rn(f0));
  }
#pragma unroll
  for (int k = 1; k < 3; ++k) {
    const float f = (float)c[k];
    const float d0 = rintf(f * (1.f / 65536.f));
    const float r = fmaf(-d0, 65536.f, f);
    const float d1 = rintf(r * (1.f / 256.f));
    o[p++] = __bfloat16_as_ushort(__float2bfloat16_rn(d0));
    o[p++] = __bfloat16_as_ushort(__float2bfloat16_rn(d1));
    o[p++] = __bfloat16_as_ushort(__float2bfloat16_rn(fmaf(-d1, 256.f, r)));
  }
}

// BF16 bit pattern of a small integer (|d| <= 255), exact.
__device__ __forceinline__ uint16_t bf16_of_int(int d) {
  if (d == 0) return 0;
  const unsigned s = d < 0 ? 0x8000u : 0u;
  const unsigned a = d < 0 ? -d : d;
  const int p = 31 - __clz(a);                    // a in [2^p, 2^(p+1))
  const unsigned man = (a << (7 - p)) & 0x7Fu;    // p <= 7
  return (uint16_t)(s | ((unsigned)(p + 127) << 7) | man);
}

// Bits of the scaled integer that S digit slices hold: nine or ten base-64 digits (54 or 60
// bits, the 1D products), seven or eight base-256 digits (55 or 62 bits, the 2D products).
__host__ __device__ constexpr int slice_bits(int S) {
  return S == 7 ? 55 : (S == 8 ? 62 : S * kBeta);
}

// round(x * 2^(bits - E)) with E = raw_max - 1022 the row exponent, by integer arithmetic
// on the FP64 fields (subnormals are flushed: they lie 2^-1022 below any row scale that
// matters here).  |result| <= 2^bits, bits <= 62.
__device__ __forceinline__ long long scaled_integer(double x, unsigned raw_max, int bits) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((u >> 52) & 0x7FF);
  if (ex == 0 || raw_max == 0) return 0;
  const long long mant = (long long)((u & ((1ULL << 52) - 1)) | (1ULL << 52));
  const int E = (int)raw_max - 1022;
  const int sh = ex - 1075 + bits - E;
  long long q;
  if (sh >= 0) {
    q = mant << sh;                     // |x| < 2^E keeps this below 2^bits
  } else if (sh > -63) {
    q = (mant + (1LL << (-sh - 1))) >> (-sh);
  } else {
    q = 0;
  }
  return (u >> 63) ? -q : q;
}

// The S digit slices of x (row exponent raw_max): dst[i * stride] = digit i, most
// significant first, in the format that S selects (slice_bits).
__device__ __forceinline__ void write_digits(double x, unsigned raw_max, int S, uint16_t *dst,
                                             long long stride) {
  long long q = scaled_integer(x, raw_max, slice_bits(S));
  if (S == 9) {
    uint16_t o[9];
    digits9(q, o);
#pragma unroll
    for (int i = 0; i < 9; ++i) dst[i * stride] = o[i];
  } else if (S == 7) {
    uint16_t o[7];
    digits256<7>(q, o);
#pragma unroll
    for (int i = 0; i < 7; ++i) dst[i * stride] = o[i];
  } else if (S == 8) {
    uint16_t o[8];
    digits256<8>(q, o);
#pragma unroll
    for (int i = 0; i < 8; ++i) dst[i * stride] = o[i];
  } else {
    for (int i = S - 1; i > 0; --i) {
      long long d = q & 63;
      if (d >= 32) d -= 64;
      dst[i * stride] = bf16_of_int((int)d);
      q = (q - d) >> kBeta;
    }
    dst[0] = bf16_of_int((int)q);
  }
}

// Row and column exponent maxima of a batch of R x C FP64 matrices (C contiguous):
// rexp[b][r] = max_c raw exponent, cexp[b][c] = max_r (either may be null).  The
// arrays must be zeroed before.  Block 32 x 8 over a 32 x 32 tile.
__global__ void k_exponents(const double *__restrict__ X, int R, int C, long long bs,
                            unsigned *__restrict__ rexp, unsigned *__restrict__ cexp) {
  if (threadIdx.x == 0 && threadIdx.y == 0) pdl_trigger();
  const int b = blockIdx.z;
  const int c = blockIdx.x * 32 + threadIdx.x;
  const int r0 = blockIdx.y * 32;
  const double *Xb = X + b * bs;
  unsigned cmax = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = r0 + threadIdx.y + 8 * j;
    const unsigned e = (r < R && c < C) ? raw_exponent(Xb[(long long)r * C + c]) : 0u;
    cmax = e > cmax ? e : cmax;
    if (rexp) {
      unsigned m = e;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
      }
      if (threadIdx.x == 0 && r < R && m) atomicMax(&rexp[(long long)b * R + r], m);
    }
  }
  if (cexp) {
    __shared__ unsigned red[8][32];
    red[threadIdx.y][threadIdx.x] = cmax;
    __syncthreads();
    if (threadIdx.y == 0) {
      unsigned m = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) m = red[k][threadIdx.x] > m ? red[k][threadIdx.x] : m;
      if (c < C && m) atomicMax(&cexp[(long long)b * C + c], m);
    }
  }
}

// Digit slices of a batch of R x C FP64 matrices:
//   natural   outN[b][i][r][c] (ld ldn)  with the row exponents rexp  (may be null)
//   transposed outT[b][i][c][r] (ld ldt) with the column exponents cexp (may be null)
// Slice i = 0 holds the most significant digit.
__global__ void k_split(const double *__restrict__ X, int R, int C, long long bs, int S,
                        const unsigned *__restrict__ rexp, uint16_t *__restrict__ outN, int ldn,
                        const unsigned *__restrict__ cexp, uint16_t *__restrict__ outT, int ldt,
                        double *__restrict__ zero_out) {
  __shared__ double tile[32][33];
  if (threadIdx.x == 0 && threadIdx.y == 0) pdl_trigger();
  pdl_wait();  // X's exponents come from the previous kernel
  const int b = blockIdx.z;
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const double *Xb = X + b * bs;
  const long long sN = (long long)R * ldn, sT = (long long)C * ldt;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = r0 + threadIdx.y + 8 * j, c = c0 + threadIdx.x;
    double x = 0.0;
    if (r < R && c < C) {
      x = Xb[(long long)r * C + c];
      // the product kernel that follows accumulates into a zeroed output of X's shape
      if (zero_out) zero_out[b * bs + (long long)r * C + c] = 0.0;
    }
    tile[threadIdx.y + 8 * j][threadIdx.x] = x;
    if (outN && r < R && c < C)
      write_digits(x, rexp[(long long)b * R + r], S,
                   outN + (long long)b * S * sN + (long long)r * ldn + c, sN);
  }
  if (!outT) return;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = c0 + threadIdx.y + 8 * j, r = r0 + threadIdx.x;
    if (r < R && c < C)
      write_digits(tile[threadIdx.x][threadIdx.y + 8 * j], cexp[(long long)b * C + c], S,
                   outT + (long long)b * S * sT + (long long)c * ldt + r, sT);
  }
}


// Exponents and digit slices of the fibers of one mode of a batch of 2D tensors (the
// contraction index of that mode's product), for a mode with stride sigma >= 32: fiber m
// of vector v holds the nk elements X[v bs + (m / sigma) nk sigma + m % sigma + i sigma],
// i < nk.  Writes the fiber's raw exponent maximum fexp[v M + m] and its S digit slices
// out[((v S + plane) M + m) ld + i] (most significant first).  Block: 256 threads over 32
// fibers (nk <= kMaxFiber); reads run across fibers (adjacent in memory), writes along
// them.  (The fibers of the fastest mode are the rows of the tensor: k_split.)
constexpr int kMaxFiber = 128;
__global__ void __launch_bounds__(256)
k_split_fibers(const double *__restrict__ X, long long bs, long long M, int nk, long long sigma,
               int S, unsigned *__restrict__ fexp, uint16_t *__restrict__ out, int ld) {
  __shared__ double tile[32][kMaxFiber + 1];
  __shared__ unsigned ex[32];
  __shared__ long long base[32];
  const int v = blockIdx.y, tid = threadIdx.x;
  const long long m0 = (long long)blockIdx.x * 32;
  const double *Xv = X + (long long)v * bs;
  if (tid < 32) {
    const long long m = m0 + tid;
    base[tid] = m < M ? (m / sigma) * (nk * sigma) + m % sigma : -1;
  }
  __syncthreads();
  {
    const int f = tid & 31;
    const long long b = base[f];
    for (int i = tid >> 5; i < nk; i += 8) tile[f][i] = b >= 0 ? Xv[b + (long long)i * sigma] : 0.0;
  }
  __syncthreads();
  if (tid < 32) {
    unsigned mx = 0;
    for (int i = 0; i < nk; ++i) {
      const unsigned r = raw_exponent(tile[tid][i]);
      mx = r > mx ? r : mx;
    }
    ex[tid] = mx;
    if (m0 + tid < M) fexp[(long long)v * M + m0 + tid] = mx;
  }
  __syncthreads();
  const long long plane = M * ld;
  for (int f = tid >> 4; f < 32; f += 16) {
    const long long m = m0 + f;
    if (m >= M) continue;
    uint16_t *row = out + ((long long)v * S) * plane + m * ld;
    for (int i = tid & 15; i < nk; i += 16) write_digits(tile[f][i], ex[f], S, row + i, plane);
  }
}

// Exponent and digit slices of the rows of a batch of [M][n] matrices (the fibers of the
// fastest mode of the 2D layout), n <= kMaxFiber, in one pass: a warp per row reads its n
// values (up to four per lane), takes the raw exponent maximum by a warp reduction, writes
// it to fexp[v M + m] and the S digit slices to out[((v S + plane) M + m) ld + i].  (The
// 1D splitter, built for the transposed pair of a 1D vector, needed a separate exponent
// pass and ran 32-wide tiles half empty on 48-value rows.)
__global__ void __launch_bounds__(256)
k_split_rows(const double *__restrict__ X, long long bs, long long M, int n, int nv, int S,
             unsigned *__restrict__ fexp, uint16_t *__restrict__ out, int ld) {
  const int lane = threadIdx.x & 31;
  const long long rows = M * nv;
  const long long plane = M * ld;
  for (long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < rows;
       row += ((long long)gridDim.x * blockDim.x) >> 5) {
    const long long v = row / M, m = row - v * M;
    const double *x = X + v * bs + m * n;
    double val[kMaxFiber / 32];
    unsigned e = 0;
#pragma unroll
    for (int h = 0; h < kMaxFiber / 32; ++h) {
      const int i = lane + 32 * h;
      val[h] = i < n ? x[i] : 0.0;
      const unsigned r = raw_exponent(val[h]);
      e = r > e ? r : e;
    }
    e = __reduce_max_sync(0xffffffffu, e);
    if (lane == 0) fexp[row] = e;
    uint16_t *dst = out + (v * S) * plane + m * ld;
#pragma unroll
    for (int h = 0; h < kMaxFiber / 32; ++h) {
      const int i = lane + 32 * h;
      if (i < n) write_digits(val[h], e, S, dst + i, plane);
    }
  }
}

// ------------------------------ the product kernel ------------------------------
struct OzArgs {
  int M, N, K;
  int SA, SB, L;                 // digit slices of A and of B, digit-pair levels kept
  int zA, zB;                    // slice-plane offset per vector (slices if per vector, 0 if shared)
  const unsigned *expA;          // raw row exponents of A [.][M], vector stride expA_bs
  long long expA_bs;
  const unsigned *expB;          // raw row exponents of B [.][N]
  long long expB_bs;
  double *out;                   // out[v * out_bs + idx(m, n)], idx = n * ldo + m, or with
  long long ldo, out_bs;         // inner > 0: (m / inner) * outer + m % inner + n * inner
  long long inner, outer;        // (the 2D mode products: m a fiber, n the mode index)
  int epi;                       // 0 store, 1 accumulate, 2 store + (V - theta_v) psi,
                                 // 3 atomic add, 4 atomic add with (V - theta_v) psi
  const double *V;               // [n * ldo + m]
  const double *psi;             // psi[v * out_bs + n * ldo + m]
  const double *theta_dev;       // theta_v (null: theta0)
  double theta0;
  int *err;                      // nonzero after a timed-out wait
  int nvec;                      // vectors (the persistent product's tile count)
};

// (hi 2^30 + lo) 2^(E - 66) rounded to the nearest FP64 value, |hi|, |lo| < 2^49: as
// (top 2^32 + 4 bot) 2^(E - 68) with top = hi + floor(lo / 2^30), bot = lo mod 2^30.
__device__ __forceinline__ double combine30(long long hi, long long lo, int E) {
  const long long top = hi + (lo >> 30);
  const long long bot4 = (lo & 0x3FFFFFFFLL) << 2;
  return b256::combine(top, bot4, E + 2);
}

// One CTA computes the 128 x kBN tile (m0, n0) of C = A B^T for vector blockIdx.z, with
// SA digit slices of A and SB of B, L levels kept: base-64 digits with L = 10 (the 1D
// products), base-256 digits with L = 8 (the 2D products).
// Warp 0 lane 0 loads (TMA), warp 1 lane 0 issues the MMAs, warp 2 owns the tensor
// memory, all four warps run the epilogue (warp w reads TMEM lanes 32w .. 32w + 31).
// The MMA issue loop is fully unrolled over the digit pairs with descriptors formed once
// per tile: a tcgen05.mma costs the issuing thread about 45 cycles at best, and at
// N = 48 any per-MMA address or loop arithmetic on that thread's critical path (a
// runtime-bounded pair loop measured about 150 cycles per MMA) idles the tensor pipe.
template <int SA, int SB, int L>
__device__ __forceinline__ void oz_tile(const CUtensorMap *tmAp, const CUtensorMap *tmBp,
                                        const OzArgs &g, int m0, int n0, int v,
                                        uint8_t *smem_raw) {
  __shared__ int abort_flag;
  const CUtensorMap &tmA = *tmAp, &tmB = *tmBp;
  uint8_t *base = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  static_assert((L == kLevels && SA + SB == kPsiSlices + kOpSlices) ||
                    (L == kLevels2 && SA == kPsiSlices2 && SB == kOpSlices2),
                "base-64 (1D) or base-256 (2D) digit products");
  static_assert(L * kBN <= (int)kTmemCols, "levels must fit in tensor memory");
  const uint32_t bstage = (uint32_t)SB * b_slice_bytes();
  uint8_t *sB = base;
  uint8_t *sA = base + kBStages * bstage;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sA + kAStages * kATileBytes);
  uint64_t *fullA = bars, *emptyA = bars + kAStages;
  uint64_t *fullB = bars + 2 * kAStages, *emptyB = fullB + kBStages;
  uint64_t *accum = emptyB + kBStages;
  uint32_t *holder = reinterpret_cast<uint32_t *>(accum + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KB = (g.K + kBK - 1) / kBK;

  if (threadIdx.x == 0) {
    pdl_trigger();
    for (int i = 0; i < kAStages; ++i) {
      tc::mbar_init(&fullA[i], 1);
      tc::mbar_init(&emptyA[i], 1);
    }
    for (int i = 0; i < kBStages; ++i) {
      tc::mbar_init(&fullB[i], 1);
      tc::mbar_init(&emptyB[i], 1);
    }
    tc::mbar_init(accum, 1);
    abort_flag = 0;
    tc::fence_barrier_init();
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
  }
  if (warp == 2) tc::tmem_alloc(holder, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *holder;
  // the set-up above overlaps the previous kernel; every global access below follows it
  pdl_wait();

  if (warp == 0 && lane == 0) {
    // ---- producer: per K block, all B slices (one stage), then the A slices one by one
    int lastA[kAStages], lastB[kBStages];
    for (int i = 0; i < kAStages; ++i) lastA[i] = -1;
    for (int i = 0; i < kBStages; ++i) lastB[i] = -1;
    bool ok = true;
    int acount = 0;
    for (int kb = 0; kb < KB && ok; ++kb) {
      const int sb = kb % kBStages;
      const uint32_t rb = (uint32_t)(kb / kBStages);
      if (!tc::mbar_wait(&emptyB[sb], (rb & 1u) ^ 1u, g.err, 1)) {
        ok = false;
        break;
      }
      tc::mbar_arrive_expect_tx(&fullB[sb], bstage);
      for (int j = 0; j < SB; ++j)
        tc::tma_load_3d(sB + sb * bstage + j * b_slice_bytes(), &tmB, &fullB[sb], kb * kBK, n0,
                        v * g.zB + j);
      lastB[sb] = (int)(rb & 1u);
      for (int i = 0; i < SA; ++i, ++acount) {
        const int sa = acount % kAStages;
        const uint32_t ra = (uint32_t)(acount / kAStages);
        if (!tc::mbar_wait(&emptyA[sa], (ra & 1u) ^ 1u, g.err, 2)) {
          ok = false;
          break;
        }
        tc::mbar_arrive_expect_tx(&fullA[sa], kATileBytes);
        tc::tma_load_3d(sA + sa * kATileBytes, &tmA, &fullA[sa], kb * kBK, m0, v * g.zA + i);
        lastA[sa] = (int)(ra & 1u);
      }
    }
    if (!ok) {
      // wind down: let every copy this thread started land before the CTA exits
      atomicExch(&abort_flag, 1);
      for (int i = 0; i < kAStages; ++i)
        if (lastA[i] >= 0) tc::mbar_wait(&fullA[i], (uint32_t)lastA[i], nullptr, 0);
      for (int i = 0; i < kBStages; ++i)
        if (lastB[i] >= 0) tc::mbar_wait(&fullB[i], (uint32_t)lastB[i], nullptr, 0);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: level l = i + j of the digit pairs accumulates at column l * kBN.
    // The first MMA of a level (K block 0, its smallest i, k-step 0) overwrites it.
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kBM, kBN);
    constexpr uint64_t kSliceStep = b_slice_bytes() >> 4;  // descriptor units (16 bytes)
    bool ok = true;
    int sa = 0;
    uint32_t pa = 0;  // A stage and its phase
    for (int kb = 0; kb < KB && ok; ++kb) {
      const int sb = kb & (kBStages - 1);
      const uint32_t rb = (uint32_t)(kb / kBStages);
      if (!tc::mbar_wait(&fullB[sb], rb & 1u, g.err, 3)) {
        ok = false;
        break;
      }
      tc::tc_fence_after();
      const uint64_t bdesc = tc::smem_desc_sw128(tc::smem_addr(sB + sb * bstage));
      const bool later = kb > 0;
#pragma unroll
      for (int i = 0; i < SA; ++i) {
        if (!tc::mbar_wait(&fullA[sa], pa, g.err, 4)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const uint64_t adesc = tc::smem_desc_sw128(tc::smem_addr(sA + sa * kATileBytes));
#pragma unroll
        for (int j = 0; j < SB; ++j) {
          if (i + j < L) {
            const bool first = i == (i + j >= SB ? i + j - SB + 1 : 0);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk)
              tc::mma_bf16(tmem + (uint32_t)((i + j) * kBN), adesc + (uint64_t)(2 * kk),
                           bdesc + (uint64_t)j * kSliceStep + (uint64_t)(2 * kk), idesc,
                           (later || kk > 0 || !first) ? 1u : 0u);
          }
        }
        tc::mma_commit(&emptyA[sa]);  // the A stage is free once these MMAs are done
        if (++sa == kAStages) {
          sa = 0;
          pa ^= 1u;
        }
      }
      if (ok) tc::mma_commit(&emptyB[sb]);
    }
    if (!ok) atomicExch(&abort_flag, 1);
    // signal the epilogue (after a failure: only so that nothing is in flight at exit)
    tc::mma_commit(accum);
  }
  __syncwarp();

  // ---- epilogue
  bool ok = tc::mbar_wait(accum, 0, g.err, 5);
  ok = __all_sync(0xffffffffu, ok);
  const int aborted = __shfl_sync(0xffffffffu, *((volatile int *)&abort_flag), 0);
  tc::tc_fence_after();
  if (ok && !aborted) {
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows) and columns of half w / 4
    const int quarter = warp & 3, half = warp >> 2;
    const int m = m0 + 32 * quarter + lane;
    const bool mvalid = m < g.M;
    const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);
    const int Em = mvalid ? (int)g.expA[v * g.expA_bs + m] - 1022 : 0;
    const bool vterm = g.epi == 2 || g.epi == 4;
    // output index of (m, n): mbase + n * nstride (one division per thread, not per output)
    const long long mbase = g.inner ? (long long)(m / g.inner) * g.outer + m % g.inner : m;
    const long long nstride = g.inner ? g.inner : g.ldo;
    const double th = vterm ? (g.theta_dev ? g.theta_dev[v] : g.theta0) : 0.0;
    static_assert(kBN % 16 == 0, "two column halves of whole 8-column groups");
    for (int c = half * (kBN / 16); c < (half + 1) * (kBN / 16); ++c) {
      long long hi[8], lo[8];
      // all levels of these 8 columns in flight at once, one wait
      uint32_t r[L][8];
#pragma unroll
      for (int l = 0; l < L; ++l) tc::tmem_ld_x8(trow + (uint32_t)(l * kBN + c * 8), r[l]);
      tc::tmem_ld_wait();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        int d[L];
#pragma unroll
        for (int l = 0; l < L; ++l) d[l] = __float2int_rn(__uint_as_float(r[l][q]));
        if (L == kLevels) {
          // levels 0..4 and 5..9 in base 64: pairs of levels fit in 32 bits (|D_l| < 2^24)
          hi[q] = (long long)(d[0] * 64 + d[1]) * (1LL << 18) +
                  (long long)(d[2] * 64 + d[3]) * 64 + d[4];
          lo[q] = (long long)(d[5] * 64 + d[6]) * (1LL << 18) +
                  (long long)(d[7] * 64 + d[8]) * 64 + d[9];
        } else {
          // levels 0..3 and 4..7 in base 256, in 64-bit arithmetic
          hi[q] = (((long long)d[0] * 256 + d[1]) * 256 + d[2]) * 256 + d[3];
          lo[q] = (((long long)d[4] * 256 + d[5]) * 256 + d[6]) * 256 + d[7];
        }
      }
      if (!mvalid) continue;
      // the group's 8 outputs: every load (V and psi for the potential term, the previous
      // value for an accumulating store) is issued before any store, so the loads' latency
      // is paid once per group, not once per output
      double val[8], ld1[8], ld2[8];
      long long idx[8];
      int En[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int n = n0 + c * 8 + q;
        idx[q] = mbase + (long long)(n < g.N ? n : n0) * nstride;
        ld1[q] = ld2[q] = 0.0;
        En[q] = n < g.N ? (int)g.expB[v * g.expB_bs + n] - 1022 : 0;
        if (n < g.N) {
          if (vterm) {
            ld1[q] = g.V[idx[q]];
            ld2[q] = g.psi[v * g.out_bs + idx[q]];
          } else if (g.epi == 1) {
            ld1[q] = g.out[v * g.out_bs + idx[q]];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int n = n0 + c * 8 + q;
        if (n >= g.N) break;
        // base 64: sum_l D_l 2^(-6 (l + 2)) = (hi 2^30 + lo) 2^(Em + En - 66), hi carrying
        // levels 0 .. 4 and lo levels 5 .. 9; base 256 (A = psi at 55 bits, B = K at 62):
        // sum_l D_l 2^(104 - 8 l) 2^(Em + En - 117) = (hi 2^32 + lo) 2^(Em + En - 69).
        // Rounded once to FP64 by integer arithmetic (GB300's FP64 pipe issues a warp
        // instruction per ~64 cycles of a sub-partition)
        val[q] = L == kLevels ? combine30(hi[q], lo[q], Em + En[q])
                              : b256::combine(hi[q], lo[q], Em + En[q] + 1);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int n = n0 + c * 8 + q;
        if (n >= g.N) break;
        double *o = g.out + v * g.out_bs + idx[q];
        const double add = vterm ? fma(ld1[q] - th, ld2[q], val[q]) : val[q];
        if (g.epi == 0 || g.epi == 2)
          *o = add;
        else if (g.epi == 1)
          *o = ld1[q] + add;
        else
          atomicAdd(o, add);  // epi 3, 4: one of exactly two terms added to a zeroed output
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 2) tc::tmem_dealloc(tmem, kTmemCols);
}

// Both products of the 1D H-apply in one launch: CTAs [0, T) compute tiles of
// C1 = K_y P^T (+ (V - theta) P), CTAs [T, 2T) tiles of C2 = P^T K_x^T, T = tiles x vectors,
// m fastest, then n, then the vector.  Each adds its tile to the zeroed output with an
// FP64 atomic: the two terms of an element are added to 0 in either order with the same
// result (0 + a is exact, and a + b = b + a), so the sum is deterministic.  One launch of
// 2T CTAs packs onto the SMs better than two of T each (T = 192 on 152 SMs at n = 512:
// each launch's second wave ran a quarter full).
__global__ void __launch_bounds__(kThreads, 1)
k_oz_gemm(const __grid_constant__ CUtensorMap tmA1, const __grid_constant__ CUtensorMap tmB1,
          const __grid_constant__ OzArgs g1, const __grid_constant__ CUtensorMap tmA2,
          const __grid_constant__ CUtensorMap tmB2, const __grid_constant__ OzArgs g2) {
  extern __shared__ uint8_t smem_raw[];
  const int tm = (g1.M + kBM - 1) / kBM, tn = (g1.N + kBN - 1) / kBN;
  const int per = (int)(gridDim.x >> 1);
  const bool second = (int)blockIdx.x >= per;
  const int r = (int)blockIdx.x - (second ? per : 0);
  const int v = r / (tm * tn), t = r % (tm * tn);
  const int m0 = (t % tm) * kBM, n0 = (t / tm) * kBN;
  if (!second)
    oz_tile<kOpSlices, kPsiSlices, kLevels>(&tmA1, &tmB1, g1, m0, n0, v, smem_raw);
  else
    oz_tile<kPsiSlices, kOpSlices, kLevels>(&tmA2, &tmB2, g2, m0, n0, v, smem_raw);
}


// One product C = A B^T (A = wave-function fiber slices, 7 base-256 digits; B = mode-matrix
// slices, 8 digits; contraction length <= 128) over tiles m fastest, then n, then the
// vector: a mode product of the 2D H-apply.  Persistent: one CTA per SM takes tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... with the three stages of a tile overlapped across
// tiles.  Warp 0 lane 0 streams the slices of tile after tile through the shared-memory
// rings; warp 1 lane 0 issues a tile's MMAs once the epilogue has released the tensor
// memory of the previous one; warps 2 .. 17 (four per TMEM lane quarter, a quarter of the
// columns each) fetch the tile's old output values while its MMAs run, then drain the
// accumulators, release the tensor memory (mbarrier tmem_empty, one arrival per epilogue
// warp) and only then store, so that the next tile's MMAs run during the stores.  (A CTA per tile, which ran the
// loads, the MMAs and the epilogue one after the other, took 5.2 ms per 8-vector apply at
// 48^4 against 3.7 ms.)
constexpr int kPEpiWarps = 16;  // four per TMEM lane quarter, a quarter of the columns each
constexpr int kPThreads = 64 + 32 * kPEpiWarps;

// The persistent kernel's epilogue (warps 2 .. 17): warp w reads TMEM lanes 32 (w % 4) ..
// + 31 (rows) and the columns of part (w - 2) / 4 of four, base-256 levels (kLevels2).
// Its per-output work is a chain of dependent integer operations, so it takes four warps
// per quarter to keep the issue slots busy (with two, a tile took 17.7 us at 21 % issue).  Per tile:
// the exponents and, for an accumulating store, the old output values are loaded before the
// accumulators are ready; after the drain the tensor memory is released, then the outputs
// are stored.
__device__ __forceinline__ void oz_epilogue_persistent(const OzArgs &g, uint32_t tmem,
                                                       uint64_t *accum, uint64_t *tmem_empty,
                                                       const int *abort_flag, long long T,
                                                       int tm, int tn) {
  constexpr int L = kLevels2;
  constexpr int NH = kBN / (kPEpiWarps / 4);  // columns per thread
  static_assert(NH % 4 == 0, "whole 4-column groups per part");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = (warp - 2) >> 2;  // half: the column part
  const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);
  const long long nstride = g.inner ? g.inner : g.ldo;
  long long tcount = 0;
  for (long long t = blockIdx.x; t < T; t += gridDim.x, ++tcount) {
    __syncwarp();  // the warp-collective loads below start converged
    const int v = (int)(t / ((long long)tm * tn)), r = (int)(t % ((long long)tm * tn));
    const int m0 = (r % tm) * kBM, n0 = (r / tm) * kBN;
    const int m = m0 + 32 * quarter + lane;
    const bool mvalid = m < g.M;
    const long long mbase = g.inner ? (long long)(m / g.inner) * g.outer + m % g.inner : m;
    const int nb = n0 + half * NH;
    // while the tile's MMAs run: the row exponent, and the values an accumulating store
    // adds to
    const int Em = mvalid ? (int)g.expA[v * g.expA_bs + m] - 1022 : 0;
    double acc[NH];
#pragma unroll
    for (int q = 0; q < NH; ++q) {
      const int n = nb + q;
      acc[q] = (g.epi == 1 && mvalid && n < g.N)
                   ? g.out[v * g.out_bs + mbase + (long long)n * nstride]
                   : 0.0;
    }
    bool ok = tc::mbar_wait(accum, (uint32_t)(tcount & 1), g.err, 5);
    ok = __all_sync(0xffffffffu, ok);
    const int aborted = __shfl_sync(0xffffffffu, *((const volatile int *)abort_flag), 0);
    if (!ok || aborted) break;
    tc::tc_fence_after();
    // the products, apart from the old values (whose loads may still be in flight), so
    // that the drain and the release do not wait for them
    double val[NH];
    // four columns at a time (eight levels each): wider groups exceed the register budget
#pragma unroll
    for (int cc = 0; cc < NH / 4; ++cc) {
      // the columns' exponents (a few cached values) load under the TMEM reads
      int En[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int n = nb + cc * 4 + q;
        En[q] = n < g.N ? (int)g.expB[v * g.expB_bs + n] - 1022 : 0;
      }
      uint32_t rr[L][4];
#pragma unroll
      for (int l = 0; l < L; ++l)
        tc::tmem_ld_x4(trow + (uint32_t)(l * kBN + half * NH + cc * 4), rr[l]);
      tc::tmem_ld_wait();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int d[L];
#pragma unroll
        for (int l = 0; l < L; ++l) d[l] = __float2int_rn(__uint_as_float(rr[l][q]));
        // (hi 2^32 + lo) 2^(Em + En - 69): levels 0..3 and 4..7 in base 256
        const long long hi = (((long long)d[0] * 256 + d[1]) * 256 + d[2]) * 256 + d[3];
        const long long lo = (((long long)d[4] * 256 + d[5]) * 256 + d[6]) * 256 + d[7];
        val[cc * 4 + q] = b256::combine(hi, lo, Em + En[q] + 1);
      }
    }
    // the accumulators are read: the next tile's MMAs may overwrite them
    tc::tc_fence_before();
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(tmem_empty);
    if (!mvalid) continue;
    if (g.epi == 2) {
      // y2: (V - theta) psi + the product, every load before any store
      const double th = g.theta_dev ? g.theta_dev[v] : g.theta0;
#pragma unroll
      for (int cc = 0; cc < NH / 4; ++cc) {
        double vv[4], pp[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int n = nb + cc * 4 + q;
          const long long idx = mbase + (long long)(n < g.N ? n : n0) * nstride;
          vv[q] = n < g.N ? g.V[idx] : 0.0;
          pp[q] = n < g.N ? g.psi[v * g.out_bs + idx] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int n = nb + cc * 4 + q;
          if (n < g.N)
            g.out[v * g.out_bs + mbase + (long long)n * nstride] =
                fma(vv[q] - th, pp[q], val[cc * 4 + q]);
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < NH; ++q) {
        const int n = nb + q;
        if (n < g.N) g.out[v * g.out_bs + mbase + (long long)n * nstride] = acc[q] + val[q];
      }
    }
  }
}

// registers are reserved per group of four warps: 18 warps take 20 warps' worth
__global__ void __launch_bounds__(kPThreads, 1)
k_oz_gemm1p(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            const __grid_constant__ OzArgs g) {
  constexpr int SA = kPsiSlices2, SB = kOpSlices2, L = kLevels2;
  extern __shared__ uint8_t smem_raw[];
  __shared__ int abort_flag;
  uint8_t *base = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t bstage = (uint32_t)SB * b_slice_bytes();
  uint8_t *sB = base;
  uint8_t *sA = base + kBStages * bstage;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sA + kAStages * kATileBytes);
  uint64_t *fullA = bars, *emptyA = bars + kAStages;
  uint64_t *fullB = bars + 2 * kAStages, *emptyB = fullB + kBStages;
  uint64_t *accum = emptyB + kBStages, *tmem_empty = accum + 1;
  uint32_t *holder = reinterpret_cast<uint32_t *>(tmem_empty + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tm = (g.M + kBM - 1) / kBM, tn = (g.N + kBN - 1) / kBN;
  const long long T = (long long)tm * tn * g.nvec;
  const int KB = (g.K + kBK - 1) / kBK;
  // one K block and one column tile (modes of at most 48 points): every tile multiplies by
  // the same B slices, loaded once into stage 0 and kept
  const bool b_fixed = KB == 1 && tn == 1;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kAStages; ++i) {
      tc::mbar_init(&fullA[i], 1);
      tc::mbar_init(&emptyA[i], 1);
    }
    for (int i = 0; i < kBStages; ++i) {
      tc::mbar_init(&fullB[i], 1);
      tc::mbar_init(&emptyB[i], 1);
    }
    tc::mbar_init(accum, 1);
    tc::mbar_init(tmem_empty, kPEpiWarps);
    abort_flag = 0;
    tc::fence_barrier_init();
    tc::prefetch_tmap(&tmA);
    tc::prefetch_tmap(&tmB);
  }
  if (warp == 1) tc::tmem_alloc(holder, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *holder;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: per tile and K block, the B slices (one stage), then the A slices
      int lastA[kAStages], lastB[kBStages];
      for (int i = 0; i < kAStages; ++i) lastA[i] = -1;
      for (int i = 0; i < kBStages; ++i) lastB[i] = -1;
      bool ok = true;
      long long acount = 0, bcount = 0;
      for (long long t = blockIdx.x; t < T && ok; t += gridDim.x) {
        const int v = (int)(t / ((long long)tm * tn)), r = (int)(t % ((long long)tm * tn));
        const int m0 = (r % tm) * kBM, n0 = (r / tm) * kBN;
        for (int kb = 0; kb < KB && ok; ++kb, ++bcount) {
          const int sb = b_fixed ? 0 : (int)(bcount % kBStages);
          const uint32_t rb = b_fixed ? 0u : (uint32_t)(bcount / kBStages);
          if (!b_fixed || t == blockIdx.x) {
            if (!tc::mbar_wait(&emptyB[sb], (rb & 1u) ^ 1u, g.err, 1)) {
              ok = false;
              break;
            }
            tc::mbar_arrive_expect_tx(&fullB[sb], bstage);
            for (int j = 0; j < SB; ++j)
              tc::tma_load_3d(sB + sb * bstage + j * b_slice_bytes(), &tmB, &fullB[sb],
                              kb * kBK, n0, v * g.zB + j);
            lastB[sb] = (int)(rb & 1u);
          }
          for (int i = 0; i < SA; ++i, ++acount) {
            const int sa = (int)(acount % kAStages);
            const uint32_t ra = (uint32_t)(acount / kAStages);
            if (!tc::mbar_wait(&emptyA[sa], (ra & 1u) ^ 1u, g.err, 2)) {
              ok = false;
              break;
            }
            tc::mbar_arrive_expect_tx(&fullA[sa], kATileBytes);
            tc::tma_load_3d(sA + sa * kATileBytes, &tmA, &fullA[sa], kb * kBK, m0,
                            v * g.zA + i);
            lastA[sa] = (int)(ra & 1u);
          }
        }
      }
      if (!ok) {
        // wind down: let every copy this thread started land before the CTA exits
        atomicExch(&abort_flag, 1);
        for (int i = 0; i < kAStages; ++i)
          if (lastA[i] >= 0) tc::mbar_wait(&fullA[i], (uint32_t)lastA[i], nullptr, 0);
        for (int i = 0; i < kBStages; ++i)
          if (lastB[i] >= 0) tc::mbar_wait(&fullB[i], (uint32_t)lastB[i], nullptr, 0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer: a tile's level l = i + j accumulates at column l * kBN; its first
      // MMA (K block 0, k-step 0, the level's smallest i) overwrites the previous tile's
      constexpr uint32_t idesc = tc::idesc_bf16_f32(kBM, kBN);
      constexpr uint64_t kSliceStep = b_slice_bytes() >> 4;
      bool ok = true;
      long long acount = 0, bcount = 0, tcount = 0;
      for (long long t = blockIdx.x; t < T && ok; t += gridDim.x, ++tcount) {
        if (tcount > 0 &&
            !tc::mbar_wait(tmem_empty, (uint32_t)((tcount - 1) & 1), g.err, 6)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        for (int kb = 0; kb < KB && ok; ++kb, ++bcount) {
          const int sb = b_fixed ? 0 : (int)(bcount % kBStages);
          const uint32_t rb = b_fixed ? 0u : (uint32_t)(bcount / kBStages);
          if (!tc::mbar_wait(&fullB[sb], rb & 1u, g.err, 3)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint64_t bdesc = tc::smem_desc_sw128(tc::smem_addr(sB + sb * bstage));
          const bool later = kb > 0;
#pragma unroll
          for (int i = 0; i < SA; ++i, ++acount) {
            const int sa = (int)(acount % kAStages);
            const uint32_t ra = (uint32_t)(acount / kAStages);
            if (!tc::mbar_wait(&fullA[sa], ra & 1u, g.err, 4)) {
              ok = false;
              break;
            }
            tc::tc_fence_after();
            const uint64_t adesc = tc::smem_desc_sw128(tc::smem_addr(sA + sa * kATileBytes));
#pragma unroll
            for (int j = 0; j < SB; ++j) {
              if (i + j < L) {
                const bool first = i == (i + j >= SB ? i + j - SB + 1 : 0);
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk)
                  tc::mma_bf16(tmem + (uint32_t)((i + j) * kBN), adesc + (uint64_t)(2 * kk),
                               bdesc + (uint64_t)j * kSliceStep + (uint64_t)(2 * kk), idesc,
                               (later || kk > 0 || !first) ? 1u : 0u);
              }
            }
            tc::mma_commit(&emptyA[sa]);  // the A stage is free once these MMAs are done
          }
          if (ok && !b_fixed) tc::mma_commit(&emptyB[sb]);
        }
        // the tile's accumulators are complete once its MMAs are (after a failure: only so
        // that nothing is in flight at exit)
        tc::mma_commit(accum);
      }
      if (!ok) atomicExch(&abort_flag, 1);
    }
  } else {
    oz_epilogue_persistent(g, tmem, accum, tmem_empty, &abort_flag, T, tm, tn);
  }
  __syncwarp();  // lanes 1 .. 31 of warps 0 and 1 wait for their lane 0
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, kTmemCols);
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

// Tensor map over a stack of BF16 slice planes [planes][rows][ld] (K = cols contiguous):
// boxes of 64 columns x box_rows rows of one plane, 128-byte swizzle, zero fill outside
// cols x rows.
bool make_slice_map(CUtensorMap *map, const void *base, int cols, int rows, long long planes,
                    int ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || (ld * 2) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * 2 * rows};
  const cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the persistent 2D product: B stages of kOpSlices2 slices and one more barrier
size_t ozp_smem_bytes() { return oz_smem_bytes(kOpSlices2) + 8; }

int round8(int n) { return (n + 7) & ~7; }

dim3 split_grid(int R, int C, int batch) { return dim3((C + 31) / 32, (R + 31) / 32, batch); }

void launch_exponents(const double *X, int R, int C, long long bs, int batch, unsigned *rexp,
                      unsigned *cexp, cudaStream_t s) {
  count_launch();
  k_exponents<<<split_grid(R, C, batch), dim3(32, 8), 0, s>>>(X, R, C, bs, rexp, cexp);
}

void launch_split(const double *X, int R, int C, long long bs, int batch, int S,
                  const unsigned *rexp, uint16_t *outN, int ldn, const unsigned *cexp,
                  uint16_t *outT, int ldt, cudaStream_t s, double *zero_out = nullptr,
                  bool dependent = false) {
  count_launch();
  if (dependent)
    launch_pdl(k_split, split_grid(R, C, batch), dim3(32, 8), 0, s, X, R, C, bs, S, rexp,
                     outN, ldn, cexp, outT, ldt, zero_out);
  else
    k_split<<<split_grid(R, C, batch), dim3(32, 8), 0, s>>>(X, R, C, bs, S, rexp, outN, ldn,
                                                            cexp, outT, ldt, zero_out);
}

// The two products of the H-apply (pass 1: A = K_y slices, B = psi slices; pass 2: A =
// psi^T slices, B = K_x slices), same output tiling, into an output zeroed beforehand.
cudaError_t launch_oz_pair(const CUtensorMap &mA1, const CUtensorMap &mB1, const OzArgs &g1,
                           const CUtensorMap &mA2, const CUtensorMap &mB2, const OzArgs &g2,
                           int nvec, cudaStream_t s) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)oz_smem_bytes(kMaxSlices));
  });
  if (attr != cudaSuccess) return attr;
  if (g1.L != kLevels || g2.L != kLevels || g1.SA != kOpSlices || g1.SB != kPsiSlices ||
      g2.SA != kPsiSlices || g2.SB != kOpSlices || g1.M != g2.M || g1.N != g2.N ||
      (g1.epi != 3 && g1.epi != 4) || (g2.epi != 3 && g2.epi != 4))
    return cudaErrorInvalidValue;
  const long long tiles = (long long)((g1.M + kBM - 1) / kBM) * ((g1.N + kBN - 1) / kBN) * nvec;
  if (2 * tiles > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
  count_launch();
  const cudaError_t le = launch_pdl(k_oz_gemm, dim3((unsigned)(2 * tiles)), dim3(kThreads),
                                          oz_smem_bytes(kMaxSlices), s, mA1, mB1, g1, mA2, mB2, g2);
  return le != cudaSuccess ? le : cudaGetLastError();
}

}  // namespace

// Tensor-core (BF16 digit) form of an operator: 1D -- slices of K_y and K_x, fixed, and a
// workspace for the slices of up to `chunk` vectors per launch; 2D -- slices of the four
// K_k, and one workspace for the fiber slices of one mode at a time.
struct TcOperator {
  int So = kOpSlices, Sp = kPsiSlices;
  int nx = 0, ny = 0, ldx = 0, ldy = 0, chunk = 0;
  uint16_t *Ky = nullptr, *Kx = nullptr;    // [So][ny][ldy], [So][nx][ldx]
  unsigned *eKy = nullptr, *eKx = nullptr;  // raw row exponents [ny], [nx]
  uint16_t *Pn = nullptr, *PT = nullptr;    // [chunk][Sp][nx][ldy], [chunk][Sp][ny][ldx]
  unsigned *eP = nullptr;                   // row exponents [chunk][nx], then column [chunk][ny]
  int *err = nullptr;                       // device flag of timed-out waits
  CUtensorMap mKy, mKx, mPn, mPT;
  // 2D: mode k has n4[k] points, stride sig4[k] in the vector layout and M4[k] = N / n4[k]
  // fibers; K4[k] [So][n][ld], fiber slices F [chunk][Sp][M4[k]][ld4[k]], exponents eF
  bool two_d = false;
  int n4[4] = {0, 0, 0, 0}, ld4[4] = {0, 0, 0, 0};
  long long M4[4] = {0, 0, 0, 0}, sig4[4] = {0, 0, 0, 0};
  uint16_t *K4[4] = {nullptr, nullptr, nullptr, nullptr};
  unsigned *eK4[4] = {nullptr, nullptr, nullptr, nullptr};
  uint16_t *F = nullptr;
  unsigned *eF = nullptr;
  CUtensorMap mK4[4], mF4[4];
};

void free_tc_operator(TcOperator *t) {
  if (!t) return;
  for (int k = 0; k < 4; ++k) {
    cudaFree(t->K4[k]);
    cudaFree(t->eK4[k]);
  }
  cudaFree(t->F);
  cudaFree(t->eF);
  cudaFree(t->Ky);
  cudaFree(t->Kx);
  cudaFree(t->eKy);
  cudaFree(t->eKx);
  cudaFree(t->Pn);
  cudaFree(t->PT);
  cudaFree(t->eP);
  cudaFree(t->err);
  delete t;
}

// The tensor-core form of a 2D operator (four modes).
cudaError_t ensure_tc_operator_2d(const DevOperator &op, cudaStream_t s) {
  TcOperator *t = new TcOperator();
  t->two_d = true;
  t->So = kOpSlices2;
  t->Sp = kPsiSlices2;
  const int So = t->So, Sp = t->Sp;
  long long maxw = 0;
  for (int k = 0; k < 4; ++k) {
    if (op.n[k] < 1 || op.n[k] > kMaxFiber) {
      delete t;
      return cudaErrorInvalidValue;
    }
    t->n4[k] = op.n[k];
    t->ld4[k] = round8(op.n[k]);
    t->M4[k] = op.N / op.n[k];
    long long sg = 1;
    for (int j = k + 1; j < 4; ++j) sg *= op.n[j];
    t->sig4[k] = sg;
    const long long w = t->M4[k] * t->ld4[k];
    maxw = w > maxw ? w : maxw;
  }
  // vectors per chunk: as many as keep the fiber-slice workspace near 1 GB
  long long ch = (1LL << 30) / (2LL * Sp * maxw);
  t->chunk = (int)(ch < 1 ? 1 : (ch > 64 ? 64 : ch));
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess && r != cudaSuccess) e = r;
  };
  for (int k = 0; k < 4; ++k) {
    chk(cudaMalloc(&t->K4[k], 2LL * So * t->n4[k] * t->ld4[k]));
    chk(cudaMalloc(&t->eK4[k], sizeof(unsigned) * t->n4[k]));
  }
  long long maxM = 0;
  for (int k = 0; k < 4; ++k) maxM = t->M4[k] > maxM ? t->M4[k] : maxM;
  chk(cudaMalloc(&t->F, 2LL * Sp * t->chunk * maxw));
  chk(cudaMalloc(&t->eF, sizeof(unsigned) * t->chunk * maxM));
  chk(cudaMalloc(&t->err, sizeof(int)));
  if (e != cudaSuccess) {
    free_tc_operator(t);
    return e;
  }
  chk(cudaMemsetAsync(t->err, 0, sizeof(int), s));
  bool ok = true;
  for (int k = 0; k < 4; ++k) {
    const int n = t->n4[k];
    chk(cudaMemsetAsync(t->eK4[k], 0, sizeof(unsigned) * n, s));
    launch_exponents(op.K[k], n, n, 0, 1, t->eK4[k], nullptr, s);
    launch_split(op.K[k], n, n, 0, 1, So, t->eK4[k], t->K4[k], t->ld4[k], nullptr, nullptr, 0, s);
    ok = ok && make_slice_map(&t->mK4[k], t->K4[k], n, n, So, t->ld4[k], kBN) &&
         make_slice_map(&t->mF4[k], t->F, n, t->M4[k], (long long)Sp * t->chunk, t->ld4[k], kBM);
  }
  chk(cudaGetLastError());
  if (e == cudaSuccess && !ok) e = cudaErrorInvalidValue;
  if (e != cudaSuccess) {
    free_tc_operator(t);
    return e;
  }
  op.tc = t;
  return cudaSuccess;
}

// Build the tensor-core form of an operator (idempotent).  Returns a cudaError_t.
cudaError_t ensure_tc_operator(const DevOperator &op, cudaStream_t s) {
  if (op.tc) return cudaSuccess;
  if (op.nmodes == 4) return ensure_tc_operator_2d(op, s);
  if (op.nmodes != 2) return cudaErrorInvalidValue;
  TcOperator *t = new TcOperator();
  t->nx = op.n[0];
  t->ny = op.n[1];
  t->ldx = round8(t->nx);
  t->ldy = round8(t->ny);
  const int So = t->So, Sp = t->Sp;
  // vectors per launch: as many as keep the slice workspace near 256 MB
  const long long per_vec = 2LL * Sp * ((long long)t->nx * t->ldy + (long long)t->ny * t->ldx);
  long long ch = (256LL << 20) / per_vec;
  t->chunk = (int)(ch < 1 ? 1 : (ch > 64 ? 64 : ch));
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess && r != cudaSuccess) e = r;
  };
  chk(cudaMalloc(&t->Ky, 2LL * So * t->ny * t->ldy));
  chk(cudaMalloc(&t->Kx, 2LL * So * t->nx * t->ldx));
  chk(cudaMalloc(&t->eKy, sizeof(unsigned) * t->ny));
  chk(cudaMalloc(&t->eKx, sizeof(unsigned) * t->nx));
  chk(cudaMalloc(&t->Pn, 2LL * Sp * t->chunk * t->nx * t->ldy));
  chk(cudaMalloc(&t->PT, 2LL * Sp * t->chunk * t->ny * t->ldx));
  chk(cudaMalloc(&t->eP, sizeof(unsigned) * t->chunk * (t->nx + t->ny)));
  chk(cudaMalloc(&t->err, sizeof(int)));
  if (e != cudaSuccess) {
    free_tc_operator(t);
    return e;
  }
  chk(cudaMemsetAsync(t->err, 0, sizeof(int), s));
  chk(cudaMemsetAsync(t->eKy, 0, sizeof(unsigned) * t->ny, s));
  chk(cudaMemsetAsync(t->eKx, 0, sizeof(unsigned) * t->nx, s));
  launch_exponents(op.K[1], t->ny, t->ny, 0, 1, t->eKy, nullptr, s);
  launch_split(op.K[1], t->ny, t->ny, 0, 1, So, t->eKy, t->Ky, t->ldy, nullptr, nullptr, 0, s);
  launch_exponents(op.K[0], t->nx, t->nx, 0, 1, t->eKx, nullptr, s);
  launch_split(op.K[0], t->nx, t->nx, 0, 1, So, t->eKx, t->Kx, t->ldx, nullptr, nullptr, 0, s);
  chk(cudaGetLastError());
  bool ok = make_slice_map(&t->mKy, t->Ky, t->ny, t->ny, So, t->ldy, kBM) &&
            make_slice_map(&t->mKx, t->Kx, t->nx, t->nx, So, t->ldx, kBN) &&
            make_slice_map(&t->mPn, t->Pn, t->ny, t->nx, (long long)Sp * t->chunk, t->ldy, kBN) &&
            make_slice_map(&t->mPT, t->PT, t->nx, t->ny, (long long)Sp * t->chunk, t->ldx, kBM);
  if (e == cudaSuccess && !ok) e = cudaErrorInvalidValue;
  if (e != cudaSuccess) {
    free_tc_operator(t);
    return e;
  }
  op.tc = t;
  return cudaSuccess;
}

// 2D H-apply (Eq. tensor_op2D): the four mode products one after the other, each as
// C[m][j] = sum_i Psi[fiber m][i] K_k[j][i] over the fibers of mode k (A = fiber slices,
// B = K_k slices); the y2 product stores its tiles with the (V - theta) Psi term, the
// other three add theirs (one CTA per output tile in each launch, so the sum is
// deterministic).
cudaError_t launch_apply_h_tc_2d(const DevOperator &op, const double *psi, double *out,
                                 int nvec, const double *theta_dev, double theta,
                                 cudaStream_t s) {
  TcOperator &t = *op.tc;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_oz_gemm1p, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ozp_smem_bytes());
  });
  if (attr != cudaSuccess) return attr;
  for (int v0 = 0; v0 < nvec; v0 += t.chunk) {
    const int nv = nvec - v0 < t.chunk ? nvec - v0 : t.chunk;
    const double *P = psi + (long long)v0 * op.N;
    double *O = out + (long long)v0 * op.N;
    for (int k = 3; k >= 0; --k) {
      const long long M = t.M4[k];
      const int n = t.n4[k];
      if (t.sig4[k] == 1) {  // the fibers are the rows of the [M][n] view
        long long blocks = (M * nv + 7) / 8;  // 8 rows (warps) per block
        if (blocks > 152LL * 16) blocks = 152LL * 16;
        count_launch();
        k_split_rows<<<(unsigned)blocks, 256, 0, s>>>(P, op.N, M, n, nv, t.Sp, t.eF, t.F,
                                                      t.ld4[k]);
      } else {
        count_launch();
        k_split_fibers<<<dim3((unsigned)((M + 31) / 32), nv), 256, 0, s>>>(
            P, op.N, M, n, t.sig4[k], t.Sp, t.eF, t.F, t.ld4[k]);
      }
      OzArgs g;
      std::memset(&g, 0, sizeof(g));
      g.L = kLevels2;
      g.M = (int)M;
      g.N = n;
      g.K = n;
      g.SA = t.Sp;
      g.SB = t.So;
      g.zA = t.Sp;
      g.zB = 0;
      g.expA = t.eF;
      g.expA_bs = M;
      g.expB = t.eK4[k];
      g.expB_bs = 0;
      g.out = O;
      g.out_bs = op.N;
      g.inner = t.sig4[k];
      g.outer = (long long)n * t.sig4[k];
      g.epi = k == 3 ? 2 : 1;
      g.V = op.V;
      g.psi = P;
      g.theta_dev = theta_dev ? theta_dev + v0 : nullptr;
      g.theta0 = theta;
      g.err = t.err;
      g.nvec = nv;
      const long long tiles = ((M + kBM - 1) / kBM) * ((n + kBN - 1) / kBN) * nv;
      if (tiles > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
      count_launch();
      // persistent: one CTA per SM (no more CTAs than tiles)
      const unsigned grid = (unsigned)(tiles < 152 ? tiles : 152);
      k_oz_gemm1p<<<grid, kPThreads, ozp_smem_bytes(), s>>>(t.mF4[k], t.mK4[k], g);
      const cudaError_t le = cudaGetLastError();
      if (le != cudaSuccess) return le;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_apply_h_tc(const DevOperator &op, const double *psi, double *out, int nvec,
                              const double *theta_dev, double theta, cudaStream_t s) {
  if (nvec <= 0) return cudaSuccess;
  cudaError_t e = ensure_tc_operator(op, s);
  if (e != cudaSuccess) return e;
  if (op.nmodes == 4) return launch_apply_h_tc_2d(op, psi, out, nvec, theta_dev, theta, s);
  TcOperator &t = *op.tc;
  const int nx = t.nx, ny = t.ny, So = t.So, Sp = t.Sp;
  for (int v0 = 0; v0 < nvec; v0 += t.chunk) {
    const int nv = nvec - v0 < t.chunk ? nvec - v0 : t.chunk;
    const double *P = psi + (long long)v0 * op.N;
    double *O = out + (long long)v0 * op.N;
    unsigned *erow = t.eP, *ecol = t.eP + (long long)t.chunk * nx;
    e = cudaMemsetAsync(t.eP, 0, sizeof(unsigned) * t.chunk * (nx + ny), s);
    if (e != cudaSuccess) return e;
    launch_exponents(P, nx, ny, op.N, nv, erow, ecol, s);
    // the split also zeroes the output, which the product kernel accumulates into; split and
    // product are launched as programmatic dependents of their predecessors
    launch_split(P, nx, ny, op.N, nv, Sp, erow, t.Pn, t.ldy, ecol, t.PT, t.ldx, s, O, true);
    OzArgs g;
    std::memset(&g, 0, sizeof(g));
    g.L = kLevels;
    g.M = ny;
    g.N = nx;
    g.out = O;
    g.ldo = ny;
    g.out_bs = op.N;
    g.err = t.err;
    // K_y P^T with the potential term: A = K_y slices (shared), B = psi slices
    g.K = ny;
    g.SA = So;
    g.SB = Sp;
    g.zA = 0;
    g.zB = Sp;
    g.expA = t.eKy;
    g.expA_bs = 0;
    g.expB = erow;
    g.expB_bs = nx;
    g.epi = 4;
    g.V = op.V;
    g.psi = P;
    g.theta_dev = theta_dev ? theta_dev + v0 : nullptr;
    g.theta0 = theta;
    // P^T K_x^T: A = psi^T slices, B = K_x slices (shared)
    OzArgs g2 = g;
    g2.K = nx;
    g2.SA = Sp;
    g2.SB = So;
    g2.zA = Sp;
    g2.zB = 0;
    g2.expA = ecol;
    g2.expA_bs = ny;
    g2.expB = t.eKx;
    g2.expB_bs = 0;
    g2.epi = 3;
    e = launch_oz_pair(t.mKy, t.mPn, g, t.mPT, t.mKx, g2, nv, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ------------------------------ failure-path self-test ------------------------------
namespace {
// Waits on an mbarrier that nothing arrives on, with the given limit: the bounded-wait
// path of the tensor-core kernels, taken on purpose.
__global__ void k_selftest_wait(long long limit, int *flag) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&bar, 1);
  tc::fence_barrier_init();
  tc::mbar_wait_for(&bar, 0, flag, 7, limit);
}
__global__ void k_selftest_touch(int *flag) {
  if (threadIdx.x == 0) flag[1] = 1;
}
}  // namespace

// Reads (synchronously) and clears the operator's timed-out-wait flag.
int tc_operator_status(const DevOperator &op) {
  if (!op.tc) return 0;
  int h = 0;
  if (cudaMemcpy(&h, op.tc->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  if (h && (cudaMemset(op.tc->err, 0, sizeof(int)) != cudaSuccess ||
            cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess))
    return -1;
  return h;
}

}  // namespace tps

extern "C" int tps_selftest_wait_timeout(int device, double seconds) {
  if (!(seconds > 0.0) || seconds > 2.0) return TPS_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return TPS_ERR_CUDA;
  int *flag = nullptr;
  if (cudaMalloc(&flag, 2 * sizeof(int)) != cudaSuccess) return TPS_ERR_NOMEM;
  int h[2] = {0, 0};
  bool ok = cudaMemset(flag, 0, 2 * sizeof(int)) == cudaSuccess;
  if (ok) {
    // SM clock cycles of the limit at the device's maximum clock (kHz attribute)
    int khz = 2000000;
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device);
    tps::count_launch();
    tps::k_selftest_wait<<<1, 32>>>((long long)(seconds * khz * 1e3), flag);
    // the device must still take work after the timed-out wait
    tps::count_launch();
    tps::k_selftest_touch<<<1, 32>>>(flag);
    ok = cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
         cudaMemcpy(h, flag, 2 * sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
  }
  cudaFree(flag);
  if (!ok || h[1] != 1) return TPS_ERR_CUDA;
  return h[0] == 7 ? TPS_ERR_TIMEOUT : TPS_ERR_CUDA;
}
