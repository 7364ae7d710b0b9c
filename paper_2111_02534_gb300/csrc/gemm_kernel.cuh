// Mode-product GEMM kernel template shared by the FP64 path (H-apply, preconditioner)
// and the FP32-arithmetic preconditioner.
//
// For every batch z:  C[z] (M x Nc) = sum over phases p of A_p[z] (M x K_p) * B_p[z] (K_p x Nc)
// followed by an epilogue (store, + (V - theta) psi, division by a Kronecker sum of
// eigenvalues, or accumulation).  Operands are row-major with unit column stride, a row
// stride and a batch stride (0 = shared), so a mode-k product of a C-ordered tensor is a
// batched GEMM with no transpose.  Two phases share one accumulator: the 1D H-apply sums
// K_x P and P K_y^T in registers.
//
// Each thread owns an R x R register tile (R = 4; R = 8 for the FP32 variants, which
// needs a quarter of the shared-memory loads per FMA); operands go through double-buffered shared
// memory, the next k-slab prefetched into registers while the current one is used.  Warps
// whose rows all lie beyond M skip the arithmetic (the parity-folded x mode has 2^k + 1
// rows, so the last row tile is nearly empty).
#pragma once

#include <cstring>
#include <mutex>
#include <unordered_map>
#include <utility>

#include "tps_internal.h"

namespace tps {
namespace gemm {

struct Opnd {
  const void *p;
  long long rs;  // row stride (elements)
  long long bs;  // batch stride (elements, 0: shared)
};

enum Epi { EPI_STORE = 0, EPI_HAPPLY = 1, EPI_DIVIDE2 = 2, EPI_ACCUM = 3, EPI_DIVIDE4 = 4 };

struct GemmArgs {
  int M, Nc, batch, nphase;
  int K[2];
  Opnd A[2], B[2];
  void *C;
  long long ldc, bsc;
  int epi;
  // EPI_HAPPLY: C += (V[(z % vmod) * vbs + m * ldv + n] - theta_z) * E[z][m][n]
  // (V and E in the accumulator's type)
  Opnd E;
  const void *V;
  long long ldv, vbs, vmod;
  const double *theta;
  long long theta_div;
  double theta0;
  // EPI_DIVIDE2: C /= (lamM[m] + lamN[n] - sigma)
  // EPI_DIVIDE4: C /= (lamM[m] + lamN[n / (n2*n3)] + lam2[(n / n3) % n2] + lam3[n % n3] - sigma)
  const void *lamM, *lamN, *lam2, *lam3;
  int n2, n3;
  double sigma;
  int tiles_m, tiles_n;
};

inline GemmArgs base_args() {
  GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.vmod = 1;
  g.theta_div = 1;
  return g;
}

constexpr int TK = 16;

template <typename Acc, typename TA, typename TB, typename TC, int TM, int TN, int R = 4>
__global__ void __launch_bounds__((TM / R) * (TN / R))
k_gemm(const GemmArgs g) {
  constexpr int NT = (TM / R) * (TN / R);
  constexpr int LA = (TM * TK + NT - 1) / NT;
  constexpr int LB = (TK * TN + NT - 1) / NT;
  __shared__ Acc As[2][TK][TM + 1];
  __shared__ Acc Bs[2][TK][TN];

  const int tid = threadIdx.x;
  const int tn = tid % (TN / R);
  const int tm = tid / (TN / R);
  const long long bid = blockIdx.x;
  const int tiles = g.tiles_m * g.tiles_n;
  const long long z = bid / tiles;
  const int t = (int)(bid % tiles);
  const int m0 = (t / g.tiles_n) * TM;
  const int n0 = (t % g.tiles_n) * TN;
  // warp-uniform: the first row any thread of this warp owns
  const int warp_tm0 = ((tid >> 5) << 5) / (TN / R);
  const bool live = m0 + warp_tm0 * R < g.M;

  Acc acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = Acc(0);

  const int ks0 = (g.K[0] + TK - 1) / TK;
  const int nstage = ks0 + (g.nphase > 1 ? (g.K[1] + TK - 1) / TK : 0);

  Acc ra[LA], rb[LB];
  auto fetch = [&](int stage) {
    const int ph = stage < ks0 ? 0 : 1;
    const int k0 = (ph == 0 ? stage : stage - ks0) * TK;
    const int Kp = g.K[ph];
    const TA *Ap = static_cast<const TA *>(g.A[ph].p) + z * g.A[ph].bs;
    const TB *Bp = static_cast<const TB *>(g.B[ph].p) + z * g.B[ph].bs;
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int e = tid + l * NT;
      const int m = e / TK, k = e % TK;
      Acc v = Acc(0);
      if (e < TM * TK && m0 + m < g.M && k0 + k < Kp)
        v = static_cast<Acc>(Ap[(long long)(m0 + m) * g.A[ph].rs + k0 + k]);
      ra[l] = v;
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int e = tid + l * NT;
      const int k = e / TN, n = e % TN;
      Acc v = Acc(0);
      if (e < TK * TN && k0 + k < Kp && n0 + n < g.Nc)
        v = static_cast<Acc>(Bp[(long long)(k0 + k) * g.B[ph].rs + n0 + n]);
      rb[l] = v;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int e = tid + l * NT;
      if (e < TM * TK) As[buf][e % TK][e / TK] = ra[l];
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int e = tid + l * NT;
      if (e < TK * TN) Bs[buf][e / TN][e % TN] = rb[l];
    }
  };

  if (nstage > 0) {
    fetch(0);
    stash(0);
  }
  __syncthreads();
  for (int s = 0; s < nstage; ++s) {
    const int buf = s & 1;
    if (s + 1 < nstage) fetch(s + 1);
    if (live) {
#pragma unroll
      for (int k = 0; k < TK; ++k) {
        Acc a[R], b[R];
#pragma unroll
        for (int i = 0; i < R; ++i) a[i] = As[buf][k][tm * R + i];
#pragma unroll
        for (int j = 0; j < R; ++j) b[j] = Bs[buf][k][tn * R + j];
#pragma unroll
        for (int i = 0; i < R; ++i)
#pragma unroll
          for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
    }
    if (s + 1 < nstage) stash(buf ^ 1);
    __syncthreads();
  }
  if (!live) return;

  double th = 0.0;
  if (g.epi == EPI_HAPPLY) th = g.theta ? g.theta[z / g.theta_div] : g.theta0;
  const Acc *lamM = static_cast<const Acc *>(g.lamM), *lamN = static_cast<const Acc *>(g.lamN);
  const Acc *lam2 = static_cast<const Acc *>(g.lam2), *lam3 = static_cast<const Acc *>(g.lam3);
  TC *Cz = static_cast<TC *>(g.C) + z * g.bsc;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int m = m0 + tm * R + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int n = n0 + tn * R + j;
      if (n >= g.Nc) continue;
      Acc c = acc[i][j];
      TC *dst = Cz + (long long)m * g.ldc + n;
      if (g.epi == EPI_HAPPLY) {
        const Acc v = static_cast<const Acc *>(g.V)[(z % g.vmod) * g.vbs + (long long)m * g.ldv + n];
        const Acc p = static_cast<const Acc *>(g.E.p)[z * g.E.bs + (long long)m * g.E.rs + n];
        c = fma(v - static_cast<Acc>(th), p, c);
      } else if (g.epi == EPI_DIVIDE2) {
        c = c / (lamM[m] + lamN[n] - static_cast<Acc>(g.sigma));
      } else if (g.epi == EPI_DIVIDE4) {
        const int n23 = g.n2 * g.n3;
        const Acc d = lamM[m] + lamN[n / n23] + lam2[(n / g.n3) % g.n2] + lam3[n % g.n3];
        c = c / (d - static_cast<Acc>(g.sigma));
      } else if (g.epi == EPI_ACCUM) {
        c += static_cast<Acc>(*dst);
      }
      *dst = static_cast<TC>(c);
    }
  }
}

// Tile choice: minimise padded work plus a one-tile-per-SM imbalance allowance,
// with a small penalty for the higher load-to-FMA ratio of small tiles.
inline void pick_tiles(const GemmArgs &g, int &tm, int &tn) {
  const int cand[3] = {32, 48, 64};
  double best = 1e300;
  tm = tn = 64;
  for (int a : cand)
    for (int b : cand) {
      const double tiles = (double)g.batch * ((g.M + a - 1) / a) * ((g.Nc + b - 1) / b);
      const double cost = (double)a * b * (tiles + 152.0) * (1.0 + 8.0 / a + 8.0 / b);
      if (cost < best) {
        best = cost;
        tm = a;
        tn = b;
      }
    }
}

template <typename Acc, typename TA, typename TB, typename TC, int TM, int TN, int R = 4>
void run(GemmArgs g, cudaStream_t s) {
  g.tiles_m = (g.M + TM - 1) / TM;
  g.tiles_n = (g.Nc + TN - 1) / TN;
  const long long blocks = (long long)g.batch * g.tiles_m * g.tiles_n;
  if (blocks <= 0) return;
  count_launch();
  k_gemm<Acc, TA, TB, TC, TM, TN, R><<<(unsigned)blocks, (TM / R) * (TN / R), 0, s>>>(g);
}

// Tile shapes: tm x tn per CTA with r x r per thread; r = 8 only for FP32 accumulation
// (an 8 x 8 FP64 tile would not fit the register budget of the FP64 variants' occupancy).
template <typename Acc, typename TA, typename TB, typename TC>
void run_tiles(const GemmArgs &g, int tm, int tn, cudaStream_t s, int r = 4) {
#define TPS_TILE_CASE(X, Y) \
  if (tm == X && tn == Y) return run<Acc, TA, TB, TC, X, Y>(g, s);
  if (r == 8 && sizeof(Acc) == 4) {
    if (tm == 128 && tn == 128) return run<Acc, TA, TB, TC, 128, 128, 8>(g, s);
    if (tm == 128 && tn == 64) return run<Acc, TA, TB, TC, 128, 64, 8>(g, s);
    if (tm == 64 && tn == 128) return run<Acc, TA, TB, TC, 64, 128, 8>(g, s);
    if (tm == 64 && tn == 64) return run<Acc, TA, TB, TC, 64, 64, 8>(g, s);
  }
  TPS_TILE_CASE(64, 64) TPS_TILE_CASE(64, 48) TPS_TILE_CASE(64, 32)
  TPS_TILE_CASE(48, 64) TPS_TILE_CASE(48, 48) TPS_TILE_CASE(48, 32)
  TPS_TILE_CASE(32, 64) TPS_TILE_CASE(32, 48) TPS_TILE_CASE(32, 32)
#undef TPS_TILE_CASE
}

// Tile autotuner.  The k-loop order of k_gemm does not depend on the tile shape, so every
// candidate computes bitwise-identical results and the choice only changes speed.  The
// first launch of a GEMM shape (precision, M, Nc, K, batch, phases) times the nine (FP32:
// thirteen) candidates with CUDA events on the caller's stream (each run twice, best kept), caches
// the fastest, and runs it; later launches of that shape use the cache.  Accumulating
// epilogues (C += ...) cannot be re-run and keep the cost-model choice, as does every
// launch while tuning is off or the stream is being captured.
struct TileKey {
  int prec, M, Nc, K0, K1, batch, nphase, epi;
  bool operator==(const TileKey &o) const { return std::memcmp(this, &o, sizeof(*this)) == 0; }
};
struct TileKeyHash {
  size_t operator()(const TileKey &k) const {
    size_t h = 1469598103934665603ULL;
    const unsigned char *p = reinterpret_cast<const unsigned char *>(&k);
    for (size_t i = 0; i < sizeof(k); ++i) h = (h ^ p[i]) * 1099511628211ULL;
    return h;
  }
};
struct TileChoice {
  int tm, tn, r;
};
struct TileCache {
  std::mutex mu;
  std::unordered_map<TileKey, TileChoice, TileKeyHash> best;
};
TileCache &tile_cache();

template <typename Acc, typename TA, typename TB, typename TC>
void gemm(GemmArgs g, cudaStream_t s) {
  int tm, tn;
  pick_tiles(g, tm, tn);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  if (!autotune_enabled() || g.epi == EPI_ACCUM || cap != cudaStreamCaptureStatusNone)
    return run_tiles<Acc, TA, TB, TC>(g, tm, tn, s);
  TileKey key{(int)sizeof(Acc) * 100 + (int)sizeof(TA) * 10 + (int)sizeof(TC), g.M, g.Nc,
              g.K[0], g.nphase > 1 ? g.K[1] : 0, g.batch, g.nphase, g.epi};
  TileCache &tc = tile_cache();
  {
    std::lock_guard<std::mutex> lock(tc.mu);
    auto it = tc.best.find(key);
    if (it != tc.best.end())
      return run_tiles<Acc, TA, TB, TC>(g, it->second.tm, it->second.tn, s, it->second.r);
  }
  // candidates: 4 x 4 register tiles on 32/48/64-wide CTA tiles; for FP32 also 8 x 8
  // register tiles on 64/128-wide CTA tiles
  TileChoice cands[13];
  int nc = 0;
  for (int a : {32, 48, 64})
    for (int b : {32, 48, 64}) cands[nc++] = {a, b, 4};
  if (sizeof(Acc) == 4)
    for (int a : {64, 128})
      for (int b : {64, 128}) cands[nc++] = {a, b, 8};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = 1e30f;
  TileChoice bestc{tm, tn, 4};
  for (int c = 0; c < nc; ++c)
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, s);
      run_tiles<Acc, TA, TB, TC>(g, cands[c].tm, cands[c].tn, s, cands[c].r);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        bestc = cands[c];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lock(tc.mu);
    tc.best[key] = bestc;
  }
  run_tiles<Acc, TA, TB, TC>(g, bestc.tm, bestc.tn, s, bestc.r);
}

// One left mode product: C[z] = A (M x M, shared) * B[z] (M x Nc), rows strided by rs.
inline GemmArgs left(const void *A, int M, const void *B, long long Nc, long long rs,
                     long long bs, void *C, int batch) {
  GemmArgs g = base_args();
  g.M = M;
  g.Nc = (int)Nc;
  g.batch = batch;
  g.nphase = 1;
  g.K[0] = M;
  g.A[0] = {A, M, 0};
  g.B[0] = {B, rs, bs};
  g.C = C;
  g.ldc = rs;
  g.bsc = bs;
  return g;
}

// One right mode product over all rows: C (rows x n) = A (rows x n) * B (n x n).
inline GemmArgs right(const void *A, long long rows, int n, const void *B, void *C) {
  GemmArgs g = base_args();
  g.M = (int)rows;
  g.Nc = n;
  g.batch = 1;
  g.nphase = 1;
  g.K[0] = n;
  g.A[0] = {A, n, 0};
  g.B[0] = {B, n, 0};
  g.C = C;
  g.ldc = n;
  g.bsc = 0;
  return g;
}

// Right product in row chunks small enough for int row counts.
template <typename Acc, typename TA, typename TB, typename TC>
void right_chunked(const TA *A, long long rows, int n, const TB *B, TC *C, cudaStream_t s) {
  const long long chunk = 1LL << 24;
  for (long long r0 = 0; r0 < rows; r0 += chunk) {
    const long long r = rows - r0 < chunk ? rows - r0 : chunk;
    gemm<Acc, TA, TB, TC>(right(A + r0 * n, r, n, B, C + r0 * n), s);
  }
}

}  // namespace gemm
}  // namespace tps
