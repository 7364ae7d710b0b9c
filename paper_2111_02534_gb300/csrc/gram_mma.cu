// FP64-accurate Gram products G = A^T B on the tensor cores: the projections of the block
// orthogonalisation and the Rayleigh-Ritz matrix of Sec. 4.1 (V^T W, W^T W, V^T H W).  A is
// nrows x p (p <= 64), B nrows x q (q <= 8), column-major, with nrows the grid's unknowns.
//
// The products are emulated by error-free digit splitting (the Ozaki scheme, as in the
// block updates, split_digits.cuh).  The contraction runs over the long index, so the
// scaling is per 64-row block: in block b, column i of A gets the exponent E_bi with
// |A[r][i]| < 2^E_bi over the block's rows and column j of B the exponent F_bj; every value
// becomes its 55-bit integer, cut into seven signed base-256 digits; the 34 digit pairs
// with i + j <= 7 are multiplied in BF16 on mma.sync (m16n8k16: M = A's columns, N = B's,
// K = 16 rows) and the pairs of one level are summed in FP32 -- exactly, since 64 terms of
// at most 196352 stay below 2^23.6.  Each block's levels are rounded once to FP64 by
// integer arithmetic and the blocks are summed in FP64.  Per block the emulation differs
// from the exact product by at most about 2^-53 (max_r |A[r][i]| sum_r |B[r][j]| + max_r
// |B[r][j]| sum_r |A[r][i]|) over the block's rows (operand truncation to 55 bits and the
// dropped levels), so with the FP64 sum of the blocks the result has the accuracy of an
// FP64 dot product, 64 rows at a time.
//
// Work: one warp per 64-row block (grid-stride).  The warp splits its block of B into
// digit fragments once and runs through A's columns 16 at a time.  Partial sums stay in
// FP64 registers per warp, then go through shared memory (per CTA) and the scratch array
// (per CTA), which the last CTA of each group of 8 and then the last group sum in a fixed
// order: the result does not depend on scheduling.
#include <cuda_runtime.h>

#include "split_digits.cuh"
#include "pdl.cuh"
#include "tps_internal.h"

namespace tps {
namespace {

using namespace b256;

constexpr int kGW = 8;        // warps per CTA
constexpr int kGRows = 64;    // rows per block: one exponent per column and block
constexpr int kGQ = 8;        // B columns (one n tile)
constexpr int kGroup = 8;     // CTAs per group of the two-level reduction
constexpr int kMaxGroups = 32;  // groups (CTAs <= kGroup kMaxGroups)

struct GramArgs {
  const double *A;
  long long lda;
  int p;
  const double *B;
  long long ldb;
  int q;
  long long nrows;
  double *G;
  int ldg;
  int trans;          // 1: store G^T (the operands were swapped so that p >= q)
  double *partial;    // gridDim.x, then ceil(gridDim.x / kGroup), x (16 MT x kGQ) sums
  unsigned *count;    // tickets: [0] groups, [1 + g] CTAs of group g; zero between calls
  const int *need;    // nullable: skip the product when *need == 0
  int vec;            // A, B, lda, ldb allow 16-byte loads of row pairs
};

__device__ __forceinline__ void mma_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                          uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The 16 values of column `col` at rows r0 + 16 ks + 2c + {0, 1, 8, 9} (ks = 0..3) into
// v[ks][e]: the rows a lane holds for the m16n8k16 fragments.  Rows past nrows and columns
// past ncol read as 0.
__device__ __forceinline__ void load_col(const double *X, long long ld, int ncol, int col,
                                         long long r0, long long nrows, int c, bool vec,
                                         double (&v)[4][4]) {
  const bool cv = col < ncol;
  const double *x = X + (long long)col * ld;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long r = r0 + 16 * ks + 2 * c + 8 * h;
      if (cv && vec && r + 1 < nrows) {
        const double2 t = __ldg(reinterpret_cast<const double2 *>(x + r));
        v[ks][2 * h] = t.x;
        v[ks][2 * h + 1] = t.y;
      } else {
        v[ks][2 * h] = (cv && r < nrows) ? __ldg(x + r) : 0.0;
        v[ks][2 * h + 1] = (cv && r + 1 < nrows) ? __ldg(x + r + 1) : 0.0;
      }
    }
}

// largest raw FP64 exponent of the column over the 64 rows (the quad of lanes holding it)
__device__ __forceinline__ unsigned col_raw_max(const double (&v)[4][4]) {
  unsigned e = 0;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)
#pragma unroll
    for (int k = 0; k < 4; ++k) e = max(e, raw_exp(v[ks][k]));
  e = max(e, __shfl_xor_sync(0xffffffffu, e, 1));
  e = max(e, __shfl_xor_sync(0xffffffffu, e, 2));
  return e;
}

// The leading NS digits of two values of one column (same exponent) as BF16 pairs.  NS = 7:
// every digit (split_digits.cuh).  NS = 3: the top digit and the two leading base-256 digits
// of the first 24-bit chunk, a 23-bit truncation (the rest, below 2^-23 of the column's
// scale, is dropped): FP32-quality products for the correction equation, which is solved
// to 1e-3 and whose result is orthonormalised in FP64.
template <int NS>
__device__ __forceinline__ void digits_n(double x0, double x1, unsigned raw_max,
                                         uint32_t (&out)[NS]) {
  if constexpr (NS == kUS) {
    digits_pair(x0, x1, raw_max, out);
  } else {
    static_assert(NS == 3, "7 or 3 digits");
    unsigned t0, a0, b0, t1, a1, b1;
    float s0, s1;
    chunks(x0, raw_max, t0, a0, b0, s0);
    chunks(x1, raw_max, t1, a1, b1, s1);
    out[0] = pack_bf16(s0 * (float)t0, s1 * (float)t1);
    const float f0 = s0 * (float)a0, f1 = s1 * (float)a1;  // |f| < 2^24: exact
    const float d00 = rintf(f0 * (1.f / 65536.f)), d01 = rintf(f1 * (1.f / 65536.f));
    out[1] = pack_bf16(d00, d01);
    out[2] = pack_bf16(rintf(fmaf(-d00, 65536.f, f0) * (1.f / 256.f)),
                       rintf(fmaf(-d01, 65536.f, f1) * (1.f / 256.f)));
  }
}

template <int MT, int NS>
__global__ void __launch_bounds__(32 * kGW, 1) k_gram_split(const GramArgs g) {
  constexpr int NL = NS == kUS ? kUL : NS;  // digit-pair levels kept: i + j < NL
  pdl_entry();
  constexpr int P = 16 * MT;  // padded A columns
  __shared__ double red[kGW][P * kGQ];
  __shared__ unsigned ticket;
  if (g.need && *g.need == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gq = lane >> 2, c = lane & 3;
  const long long nblk = (g.nrows + kGRows - 1) / kGRows;
  double acc[MT][4];
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int t = 0; t < 4; ++t) acc[mt][t] = 0.0;

  for (long long blk = (long long)blockIdx.x * kGW + warp; blk < nblk;
       blk += (long long)gridDim.x * kGW) {
    const long long r0 = blk * kGRows;
    // B: column gq, its exponent and digit fragments {k 2c, 2c+1 | 2c+8, 2c+9; col gq}
    uint32_t bf[NS][4][2];
    unsigned f0, f1;
    {
      double bv[4][4];
      load_col(g.B, g.ldb, g.q, gq, r0, g.nrows, c, g.vec, bv);
      const unsigned fb = col_raw_max(bv);
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t d[NS];
          digits_n<NS>(bv[ks][2 * h], bv[ks][2 * h + 1], fb, d);
#pragma unroll
          for (int j = 0; j < NS; ++j) bf[j][ks][h] = d[j];
        }
      // exponents of this lane's output columns 2c and 2c + 1
      f0 = __shfl_sync(0xffffffffu, fb, (2 * c) * 4);
      f1 = __shfl_sync(0xffffffffu, fb, (2 * c + 1) * 4);
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      // A: columns 16 mt + gq (fragment rows g) and + 8 (rows g + 8)
      // when the m tile's upper 8 columns are all past p (p <= 8, or a ragged last tile),
      // the warp skips them: zero fragments, no loads, no splitting
      const bool upper = 16 * mt + 8 < g.p;
      double av[2][4][4];
      load_col(g.A, g.lda, g.p, 16 * mt + gq, r0, g.nrows, c, g.vec, av[0]);
      if (upper) load_col(g.A, g.lda, g.p, 16 * mt + gq + 8, r0, g.nrows, c, g.vec, av[1]);
      const unsigned e0 = col_raw_max(av[0]), e1 = upper ? col_raw_max(av[1]) : 0u;
      float lv[NL][4];
#pragma unroll
      for (int l = 0; l < NL; ++l)
#pragma unroll
        for (int t = 0; t < 4; ++t) lv[l][t] = 0.f;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        // A fragment regs: {i g, k 2c..}, {i g+8, k 2c..}, {i g, k 2c+8..}, {i g+8, k 2c+8..}
        uint32_t af[NS][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int col = r & 1, h = r >> 1;
          if (col && !upper) {
#pragma unroll
            for (int i = 0; i < NS; ++i) af[i][r] = 0u;
            continue;
          }
          uint32_t d[NS];
          digits_n<NS>(av[col][ks][2 * h], av[col][ks][2 * h + 1], col ? e1 : e0, d);
#pragma unroll
          for (int i = 0; i < NS; ++i) af[i][r] = d[i];
        }
#pragma unroll
        for (int j = 0; j < NS; ++j)
#pragma unroll
          for (int i = 0; i < NS; ++i)
            if (i + j < NL) mma_16816(lv[i + j], af[i], bf[j][ks][0], bf[j][ks][1]);
      }
      // levels -> FP64: value = (hi 2^32 + lo) 2^(E + F - 70) (Horner in base 256, levels
      // 0..3 and 4..7); C fragment t: column 16 mt + gq + 8 (t >> 1) of A, 2c + (t & 1) of B
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        long long hi = 0, lo = 0;
#pragma unroll
        for (int l = 0; l < kUL; ++l) {  // levels NL .. 7 are zero
          const long long dl = l < NL ? (long long)__float2int_rn(lv[l < NL ? l : 0][t]) : 0;
          if (l < kUL / 2)
            hi = hi * 256 + dl;
          else
            lo = lo * 256 + dl;
        }
        const unsigned er = (t & 2) ? e1 : e0, fr = (t & 1) ? f1 : f0;
        if (er && fr) acc[mt][t] += combine(hi, lo, (int)er - 1022 + (int)fr - 1022);
      }
    }
  }

  // per CTA: the warps' sums in shared memory, added in warp order
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int t = 0; t < 4; ++t)
      red[warp][(16 * mt + gq + 8 * (t >> 1)) * kGQ + 2 * c + (t & 1)] = acc[mt][t];
  __syncthreads();
  constexpr int E = P * kGQ;
  double *part = g.partial + (long long)blockIdx.x * E;
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kGW; ++w) s += red[w][e];
    part[e] = s;
  }
  // Two-level reduction over the CTAs, in a fixed order: the last CTA of each group of
  // kGroup adds the group's partial sums, the last group adds the group sums.  Every
  // thread issues all its loads of a level before adding them.
  const int ngroups = (gridDim.x + kGroup - 1) / kGroup;
  const int grp = blockIdx.x / kGroup;
  const int gsize = min(kGroup, (int)gridDim.x - grp * kGroup);
  __threadfence();  // this CTA's sums are visible before its ticket is taken
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(g.count + 1 + grp, 1u);
  __syncthreads();
  if (ticket != (unsigned)(gsize - 1)) return;
  __threadfence();
  double *gpart = g.partial + (long long)gridDim.x * E + (long long)grp * E;
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    const double *src = g.partial + (long long)grp * kGroup * E + e;
    double v[kGroup];
#pragma unroll
    for (int b = 0; b < kGroup; ++b) v[b] = b < gsize ? __ldcg(src + (long long)b * E) : 0.0;
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < kGroup; ++b) s += v[b];
    gpart[e] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    g.count[1 + grp] = 0u;  // re-armed for the next call on this stream
    ticket = atomicAdd(g.count, 1u);
  }
  __syncthreads();
  if (ticket != (unsigned)(ngroups - 1)) return;
  __threadfence();
  const double *gbase = g.partial + (long long)gridDim.x * E;
  for (int e = threadIdx.x; e < g.p * g.q; e += blockDim.x) {
    const int i = e % g.p, j = e / g.p;
    const double *src = gbase + i * kGQ + j;
    double v[kMaxGroups];
#pragma unroll
    for (int b = 0; b < kMaxGroups; ++b) v[b] = b < ngroups ? __ldcg(src + (long long)b * E) : 0.0;
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < kMaxGroups; ++b) s += v[b];
    if (g.trans)
      g.G[(long long)i * g.ldg + j] = s;
    else
      g.G[(long long)j * g.ldg + i] = s;
  }
  if (threadIdx.x == 0) *g.count = 0u;
}

int sm_count_cached() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      n = v;
  }
  return n > 0 ? n : 1;
}

}  // namespace

bool gram_split_supported(int p, int q, int batch) {
  const int lo = p < q ? p : q, hi = p < q ? q : p;
  return batch == 1 && lo >= 1 && lo <= kGQ && hi <= 64;
}

bool gram_split_pays(int p, int q) { return p * q >= 32; }

void launch_gram_split(const double *A, long long lda, int p, const double *B, long long ldb,
                       int q, long long nrows, double *G, int ldg, GramScratch &scr,
                       cudaStream_t s, const int *need, bool low) {
  if (p <= 0 || q <= 0) return;
  int trans = 0;
  if (p < q) {  // G^T = B^T A: the narrower operand is B
    std::swap(A, B);
    std::swap(lda, ldb);
    std::swap(p, q);
    trans = 1;
  }
  GramArgs g;
  g.A = A;
  g.lda = lda;
  g.p = p;
  g.B = B;
  g.ldb = ldb;
  g.q = q;
  g.nrows = nrows;
  g.G = G;
  g.ldg = ldg;
  g.trans = trans;
  g.partial = scr.partial;
  g.count = scr.count;
  g.need = need;
  g.vec = ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) == 0 &&
          (lda & 1) == 0 && (ldb & 1) == 0;
  const int MT = (p + 15) / 16;
  const long long nblk = (nrows + kGRows - 1) / kGRows;
  long long grid = (nblk + kGW - 1) / kGW;
  // partial sums of the CTAs and of their groups fit the scratch
  const long long cap = scr.capacity / (16LL * MT * kGQ) * kGroup / (kGroup + 1);
  grid = grid < sm_count_cached() ? grid : sm_count_cached();
  grid = grid < cap ? grid : cap;
  grid = grid < kGroup * kMaxGroups ? grid : kGroup * kMaxGroups;
  if (grid < 1) grid = 1;
  count_launch();
  if (low) {
    switch (MT) {
      case 1: launch_pdl(k_gram_split<1, 3>, (unsigned)grid, 32 * kGW, 0, s, g); break;
      case 2: launch_pdl(k_gram_split<2, 3>, (unsigned)grid, 32 * kGW, 0, s, g); break;
      case 3: launch_pdl(k_gram_split<3, 3>, (unsigned)grid, 32 * kGW, 0, s, g); break;
      default: launch_pdl(k_gram_split<4, 3>, (unsigned)grid, 32 * kGW, 0, s, g); break;
    }
    return;
  }
  switch (MT) {
    case 1: launch_pdl(k_gram_split<1, kUS>, (unsigned)grid, 32 * kGW, 0, s, g); break;
    case 2: launch_pdl(k_gram_split<2, kUS>, (unsigned)grid, 32 * kGW, 0, s, g); break;
    case 3: launch_pdl(k_gram_split<3, kUS>, (unsigned)grid, 32 * kGW, 0, s, g); break;
    default: launch_pdl(k_gram_split<4, kUS>, (unsigned)grid, 32 * kGW, 0, s, g); break;
  }
}

}  // namespace tps
