// Block Jacobi-Davidson eigensolver (Sec. 4.1) with the fast-diagonalisation
// preconditioner of Sec. 4.2, for the lowest eigenpairs of the symmetric Kronecker-sum
// Hamiltonian.  For symmetric H the Newton system of Eq. jdqr reduces to Ritz pairs of
// V^T H V and the correction equation Eq. jdcor; the paper's single-vector JDQR is
// block size 1.
//
// All vector work runs in device kernels on one stream.  The host keeps the loop
// state (basis size, number of locked pairs) and reads a handful of scalars per
// outer iteration (Ritz values, residual norms, rank flags) to steer it.
//
// 1D problems in a heavy-exchange sector run on the parity-folded operator (Sec. 5.1,
// parity selection rule): half the x grid, roughly 2.6x fewer flops per H-apply.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "jd_kernels.h"
#include "tps_internal.h"

namespace tps {

// Optional device timing of the operator applications: CUDA events bracket every H and
// preconditioner launch group on the solve's stream; completed pairs are drained at the
// host synchronisation points of the outer loop.
struct PhaseTiming {
  bool on = false;
  std::vector<cudaEvent_t> all, free_ev;
  // kinds: 0 FP64 H, 1 preconditioner, 2 FP32 H, 3 Gram products, 4 block updates, 5
  // Rayleigh-Ritz eigensolves.  The skinny kinds (hundreds of short launches per solve)
  // and the Ritz solves are timed on every kSample-th launch only: their flops, bytes and
  // time then refer to the sampled launches, and launches[] counts all of them
  static constexpr int kKinds = 6;
  static constexpr int kSample = 4;
  long long seen[kKinds] = {0, 0, 0, 0, 0, 0};
  long long timed[kKinds] = {0, 0, 0, 0, 0, 0};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pend[kKinds];
  double ms[kKinds] = {0, 0, 0, 0, 0, 0}, flops[kKinds] = {0, 0, 0, 0, 0, 0};
  double bytes[kKinds] = {0, 0, 0, 0, 0, 0};
  long long launches[kKinds] = {0, 0, 0, 0, 0, 0};
  void reset(bool enable) {
    on = enable;
    for (int k = 0; k < kKinds; ++k) {
      ms[k] = flops[k] = bytes[k] = 0.0;
      launches[k] = seen[k] = timed[k] = 0;
    }
  }
  cudaEvent_t get() {
    if (free_ev.empty()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      all.push_back(e);
      return e;
    }
    cudaEvent_t e = free_ev.back();
    free_ev.pop_back();
    return e;
  }
  void drain() {
    for (int k = 0; k < kKinds; ++k) {
      for (auto &pr : pend[k]) {
        cudaEventSynchronize(pr.second);
        float t = 0.f;
        if (cudaEventElapsedTime(&t, pr.first, pr.second) == cudaSuccess) ms[k] += t;
        free_ev.push_back(pr.first);
        free_ev.push_back(pr.second);
      }
      pend[k].clear();
    }
  }
  void destroy() {
    for (auto e : all) cudaEventDestroy(e);
    all.clear();
    free_ev.clear();
  }
};

struct SolverWorkspace {
  PhaseTiming tm;
  int prec_dtype = TPS_F64;  // arithmetic of the preconditioner applications
  bool corr_low = false;     // FP32-arithmetic Gram/update products in the correction solve
  int h64_dtype = TPS_F64;   // FP64 H-applies on the FMA pipe or the tensor cores
  long long N = 0;
  int mmax = 0, b = 0, kmax = 0, steps = 0;
  double *arena = nullptr;
  size_t arena_bytes = 0;
  // big vectors
  double *V = nullptr, *HV = nullptr, *V2 = nullptr, *HV2 = nullptr;  // [mmax][N]
  double *QX = nullptr, *KQX = nullptr;                                // [kmax + b][N]
  double *HX = nullptr, *R = nullptr, *P = nullptr, *W = nullptr;      // [b][N]
  double *Z = nullptr;                                                 // [(steps+1) b][N]
  double *T2 = nullptr;                                                // [b][N] scratch
  // small
  double *G = nullptr, *Y = nullptr;            // [mmax * mmax]
  double *Arot = nullptr;                       // [mmax * mmax] Y^T G Y of the last Ritz solve
  double *theta = nullptr, *theta2 = nullptr;   // [mmax]
  double *nrm2 = nullptr, *ref = nullptr;       // [max(b, kmax + b)]
  double *C = nullptr;                          // [(kmax + mmax + b) * b] projection coefficients
  double *Mq = nullptr, *Minv = nullptr;        // [(kmax+b)^2]
  double *Rinv = nullptr;                       // [b * b]
  int *keep = nullptr;                          // [b]
  int *keep0 = nullptr;                         // [b] first Cholesky-QR pass (graph solver)
  int *gstate = nullptr;                        // graph solver: converged flag, iterations
  double *gshift = nullptr;                     // graph solver: the preconditioner's shift
  cudaStream_t capture = nullptr;               // graph solver: private stream for capture (the
                                                // legacy default stream cannot capture)
  int *jstat = nullptr;                         // Jacobi sweeps, rotating rounds, calls
  int *dgks = nullptr;                          // second-pass flag, passes needed, decisions
  GmresState gm;
  double *h_pinned = nullptr;                   // host readback buffer
  int *hi_pinned = nullptr;
};

namespace {

// Timers of the running solve (tps_solver_opts.timing), for the skinny-kernel wrappers.
thread_local PhaseTiming *tl_timing = nullptr;
thread_local bool tl_split_updates = false;  // FP64 updates as digit-split tensor-core products
thread_local bool tl_split_grams = false;    // FP64 Grams as digit-split tensor-core products

// launch_gram / launch_update with CUDA-event timing and algorithmic work counts
// low: FP32-arithmetic products (the correction equation's); like conditional launches
// (need, which may do nothing) they are neither timed nor counted in the FP64 Gram and
// update statistics
void tgram(const double *A, long long lda, long long bsa, int p, const double *B, long long ldb,
           long long bsb, int q, long long nrows, double *G, int ldg, long long bsg, int batch,
           GramScratch &scr, cudaStream_t s, const int *need = nullptr, bool low = false) {
  PhaseTiming *t = tl_timing;
  const bool live = !need && !low && t && t->on && p > 0 && q > 0 && batch > 0 && nrows > 0;
  if (live) t->launches[3] += 1;
  const bool rec = live && (t->seen[3]++ % PhaseTiming::kSample) == 0;
  cudaEvent_t a = nullptr, b = nullptr;
  if (rec) {
    a = t->get();
    b = t->get();
    cudaEventRecord(a, s);
  }
  // as for the updates, the split pays on tall blocks only
  if (tl_split_grams && nrows >= 100000 && gram_split_supported(p, q, batch) &&
      gram_split_pays(p, q))
    launch_gram_split(A, lda, p, B, ldb, q, nrows, G, ldg, scr, s, need, low);
  else
    launch_gram(A, lda, bsa, p, B, ldb, bsb, q, nrows, G, ldg, bsg, batch, scr, s, need, low);
  if (rec) {
    cudaEventRecord(b, s);
    t->pend[3].push_back({a, b});
    t->flops[3] += 2.0 * nrows * p * q * batch;
    t->bytes[3] += 8.0 * nrows * (p + q) * batch;
  }
}

void tupdate(const double *A, long long lda, long long bsa, int p, const double *Y, int ldy,
             long long bsy, int q, double alpha, double beta, double *C, long long ldc,
             long long bsc, long long nrows, int batch, cudaStream_t s,
             const int *need = nullptr, bool low = false, bool split_ok = true) {
  PhaseTiming *t = tl_timing;
  const bool live = !need && !low && t && t->on && p > 0 && q > 0 && batch > 0 && nrows > 0;
  if (live) t->launches[4] += 1;
  const bool rec = live && (t->seen[4]++ % PhaseTiming::kSample) == 0;
  cudaEvent_t a = nullptr, b = nullptr;
  if (rec) {
    a = t->get();
    b = t->get();
    cudaEventRecord(a, s);
  }
  // the split pays on tall blocks: at the sweep's sizes (n <= 384, fewer than 10^5 rows
  // per sector) its fixed per-row work made the 256-instance sweep 7 % slower than FMA
  if (!low && split_ok && tl_split_updates && nrows * batch >= 100000 && p >= 8)
    launch_update_split(A, lda, bsa, p, Y, ldy, bsy, q, alpha, beta, C, ldc, bsc, nrows, batch, s,
                        need);
  else
    launch_update(A, lda, bsa, p, Y, ldy, bsy, q, alpha, beta, C, ldc, bsc, nrows, batch, s, need,
                  low);
  if (rec) {
    cudaEventRecord(b, s);
    t->pend[4].push_back({a, b});
    t->flops[4] += 2.0 * nrows * p * q * batch;
    t->bytes[4] += 8.0 * nrows * (p + (beta != 0.0 ? 2 : 1) * q) * batch;
  }
}

struct Ctx {
  tps_ctx *ctx;
  const DevOperator &op;
  SolverWorkspace &w;
  cudaStream_t s;
  long long N;
};

// ncols random start columns, made on the device (counter-based, so reproducible)
int fill_random(Ctx &c, double *dst, int ncols, uint64_t seed, uint64_t &counter) {
  const long long n = (long long)ncols * c.N;
  launch_fill_normal(dst, n, seed, counter, c.s);
  counter += (uint64_t)n + 1;
  TPS_CUDA_TRY(c.ctx, cudaGetLastError());
  return TPS_OK;
}

// algorithmic FP64 flops of one H application (sum over modes of 2 N n_k, plus 3 N for
// the pointwise (V - theta) psi term) and of one preconditioner application (forward and
// backward mode products, 4 N n_k, plus N divisions)
double h_flops_per_vec(const DevOperator &op) {
  double s = 0.0;
  for (int k = 0; k < op.nmodes; ++k) s += op.n[k];
  return 2.0 * op.N * s + 3.0 * op.N;
}
double prec_flops_per_vec(const DevOperator &op) {
  double s = 0.0;
  for (int k = 0; k < op.nmodes; ++k) s += op.n[k];
  return 4.0 * op.N * s + (double)op.N;
}

void apply_h_timed(Ctx &c, const double *in, double *out, int nvec, const double *theta,
                   bool low) {
  PhaseTiming &t = c.w.tm;
  const int kind = low ? 2 : 0;
  cudaEvent_t a = nullptr, b = nullptr;
  if (t.on) {
    a = t.get();
    b = t.get();
    cudaEventRecord(a, c.s);
  }
  if (low)
    launch_apply_h_f32(c.op, in, out, nvec, theta, 0.0, c.ctx->ws, c.s);
  else if (c.w.h64_dtype == TPS_F64_TC)
    launch_apply_h_tc(c.op, in, out, nvec, theta, 0.0, c.s);  // errors surface at the next sync
  else
    launch_apply_h(c.op, in, out, nvec, theta, 0.0, c.s);
  if (t.on) {
    cudaEventRecord(b, c.s);
    t.pend[kind].push_back({a, b});
  }
  t.flops[kind] += nvec * h_flops_per_vec(c.op);
  t.launches[kind] += 1;
}

void apply_prec_timed(Ctx &c, const double *in, double *out, int nvec, double shift,
                      const double *shift_dev = nullptr) {
  PhaseTiming &t = c.w.tm;
  cudaEvent_t a = nullptr, b = nullptr;
  if (t.on) {
    a = t.get();
    b = t.get();
    cudaEventRecord(a, c.s);
  }
  if (c.w.prec_dtype == TPS_TF32_TC)
    launch_apply_prec_tf32(c.op, in, out, nvec, shift, c.ctx->ws, c.s, shift_dev);
  else if (c.w.prec_dtype == TPS_F32)
    launch_apply_prec_f32(c.op, in, out, nvec, shift, c.ctx->ws, c.s);
  else
    launch_apply_prec(c.op, in, out, nvec, shift, c.ctx->ws, c.s);
  if (t.on) {
    cudaEventRecord(b, c.s);
    t.pend[1].push_back({a, b});
  }
  t.flops[1] += nvec * prec_flops_per_vec(c.op);
  t.launches[1] += 1;
}

// diag(A^T A) for ncols columns -> out[ncols] (device)
void col_norms2(Ctx &c, const double *A, int ncols, double *out) {
  launch_col_norms2(A, c.N, ncols, c.N, out, c.ctx->gscr, c.s);
}

// T (b cols) <- orthonormal basis of span(T) minus span(B1, B2); B1, B2 orthonormal blocks
// (nb1, nb2 columns, ld N).  Returns the number of kept columns (moved to the front).
int orthonormalize(Ctx &c, const double *B1, int nb1, const double *B2, int nb2, double *T, int b,
                   int *rank) {
  SolverWorkspace &w = c.w;
  col_norms2(c, T, b, w.ref);
  // block classical Gram-Schmidt; the second pass runs only where the first lost more
  // than half of a column's squared norm (the DGKS criterion), decided on the device
  for (int pass = 0; pass < 2 && nb1 + nb2 > 0; ++pass) {
    const int *need = nullptr;
    if (pass == 1) {
      col_norms2(c, T, b, w.nrm2);
      launch_dgks_flag(w.ref, w.nrm2, b, w.dgks, w.dgks + 1, c.s);
      need = w.dgks;
    }
    if (nb1 > 0) {
      tgram(B1, c.N, 0, nb1, T, c.N, 0, b, c.N, w.C, nb1, 0, 1, c.ctx->gscr, c.s, need);
      tupdate(B1, c.N, 0, nb1, w.C, nb1, 0, b, -1.0, 1.0, T, c.N, 0, c.N, 1, c.s, need);
    }
    if (nb2 > 0) {
      tgram(B2, c.N, 0, nb2, T, c.N, 0, b, c.N, w.C, nb2, 0, 1, c.ctx->gscr, c.s, need);
      tupdate(B2, c.N, 0, nb2, w.C, nb2, 0, b, -1.0, 1.0, T, c.N, 0, c.N, 1, c.s, need);
    }
  }
  // Cholesky QR twice; the first pass drops numerically dependent columns
  for (int pass = 0; pass < 2; ++pass) {
    tgram(T, c.N, 0, b, T, c.N, 0, b, c.N, w.C, b, 0, 1, c.ctx->gscr, c.s);
    launch_chol_inv(w.C, b, pass == 0 ? w.ref : nullptr, pass == 0 ? 1e-7 : 1e-12, w.Rinv,
                    w.keep, c.s);
    // T Rinv stays on the FMA pipe: T's columns can differ in norm by many orders (nearly
    // dependent directions), which a row-scaled digit split would resolve only relative to
    // the largest column of each row
    tupdate(T, c.N, 0, b, w.Rinv, b, 0, b, 1.0, 0.0, w.T2, c.N, 0, c.N, 1, c.s, nullptr, false,
            false);
    TPS_CUDA_TRY(c.ctx, cudaMemcpyAsync(T, w.T2, (size_t)b * c.N * sizeof(double),
                                        cudaMemcpyDeviceToDevice, c.s));
    if (pass == 0) {
      TPS_CUDA_TRY(c.ctx, cudaMemcpyAsync(w.hi_pinned, w.keep, b * sizeof(int),
                                          cudaMemcpyDeviceToHost, c.s));
    }
  }
  TPS_CUDA_TRY(c.ctx, cudaStreamSynchronize(c.s));
  TPS_CUDA_TRY(c.ctx, cudaGetLastError());
  int r = 0;
  for (int j = 0; j < b; ++j) {
    if (w.hi_pinned[j]) {
      if (r != j)
        TPS_CUDA_TRY(c.ctx, cudaMemcpyAsync(T + (long long)r * c.N, T + (long long)j * c.N,
                                            c.N * sizeof(double), cudaMemcpyDeviceToDevice, c.s));
      ++r;
    }
  }
  *rank = r;
  return TPS_OK;
}

// Out = Kt^-1 Y for nsys columns: projected preconditioner (use_prec) or projector.
void kt_inverse(Ctx &c, const double *Qt, int nq, const double *KQt, int use_prec, double shift,
                const double *Yin, int nsys, double *Out, const double *shift_dev = nullptr) {
  SolverWorkspace &w = c.w;
  if (use_prec) {
    apply_prec_timed(c, Yin, Out, nsys, shift, shift_dev);
    if (nq > 0) {
      tgram(Qt, c.N, 0, nq, Out, c.N, 0, nsys, c.N, w.C, nq, 0, 1, c.ctx->gscr, c.s, nullptr,
            w.corr_low);
      // C2 = Minv * C, stored after C
      double *C2 = w.C + (long long)nq * nsys;
      launch_small_gemm(nq, nsys, nq, 1.0, w.Minv, nq, w.C, nq, 0.0, C2, nq, c.s);
      tupdate(KQt, c.N, 0, nq, C2, nq, 0, nsys, -1.0, 1.0, Out, c.N, 0, c.N, 1, c.s, nullptr,
              w.corr_low);
    }
  } else {
    if (Out != Yin) launch_axpby_cols(nsys, c.N, 1.0, Yin, c.N, 0.0, Out, c.N, c.s);
    for (int pass = 0; pass < 2 && nq > 0; ++pass) {
      tgram(Qt, c.N, 0, nq, Out, c.N, 0, nsys, c.N, w.C, nq, 0, 1, c.ctx->gscr, c.s, nullptr,
            w.corr_low);
      tupdate(Qt, c.N, 0, nq, w.C, nq, 0, nsys, -1.0, 1.0, Out, c.N, 0, c.N, 1, c.s, nullptr,
              w.corr_low);
    }
  }
}

int alloc_workspace(tps_ctx *ctx, long long N, int mmax, int b, int kmax, int steps) {
  SolverWorkspace *w = ctx->sw;
  if (w && w->N == N && w->mmax >= mmax && w->b >= b && w->kmax >= kmax && w->steps >= steps)
    return TPS_OK;
  if (w) {
    mmax = std::max(mmax, w->mmax);
    b = std::max(b, w->b);
    kmax = std::max(kmax, w->kmax);
    steps = std::max(steps, w->steps);
    free_solver_workspace(ctx);
  }
  w = new SolverWorkspace;
  ctx->sw = w;
  w->N = N;
  w->mmax = mmax;
  w->b = b;
  w->kmax = kmax;
  w->steps = steps;
  const int mk2 = std::max(mmax, kmax);  // V2/HV2 also hold the final H Q and residuals
  const int bw = std::max(b, kmax);       // widest block orthonormalised (refinement start)
  const long long nbig = 2LL * mmax + 2LL * mk2 + 2LL * (kmax + b) + 4LL * b +
                         (long long)(steps + 1) * b + bw;
  const int q = kmax + b;
  const long long nsmall = 3LL * mmax * mmax + 2LL * mmax + 2LL * std::max(q, mmax) +
                           2LL * (q + mmax + b) * std::max(b, q) + 2LL * q * q + (long long)bw * bw + bw +
                           /* gmres */ (long long)b * ((steps + 1) * steps + 2 * steps + (steps + 1) +
                                                      3 + steps + (steps + 1)) + 64 +
                           /* keep0, graph state, shift */ 2LL * bw + 96;
  const size_t bytes = ((size_t)nbig * N + (size_t)nsmall) * sizeof(double) + 4096 * 4;
  TPS_CUDA_TRY(ctx, cudaMalloc((void **)&w->arena, bytes));
  w->arena_bytes = bytes;
  double *p = w->arena;
  auto take = [&](long long n) {
    double *r = p;
    p += (n + 31) / 32 * 32;
    return r;
  };
  w->V = take((long long)mmax * N);
  w->HV = take((long long)mmax * N);
  w->V2 = take((long long)mk2 * N);
  w->HV2 = take((long long)mk2 * N);
  w->QX = take((long long)q * N);
  w->KQX = take((long long)q * N);
  w->HX = take((long long)b * N);
  w->R = take((long long)b * N);
  w->P = take((long long)b * N);
  w->W = take((long long)b * N);
  w->Z = take((long long)(steps + 1) * b * N);
  w->T2 = take((long long)bw * N);
  w->G = take((long long)mmax * mmax);
  w->Y = take((long long)mmax * mmax);
  w->Arot = take((long long)mmax * mmax);
  w->theta = take(mmax);
  w->theta2 = take(mmax);
  w->nrm2 = take(std::max(q, mmax));
  w->ref = take(std::max(q, mmax));
  w->C = take(2LL * (q + mmax + b) * std::max(b, q));
  w->Mq = take((long long)q * q);
  w->Minv = take((long long)q * q);
  w->Rinv = take((long long)bw * bw);
  w->gm.Hb = take((long long)b * (steps + 1) * steps);
  w->gm.cs = take((long long)b * steps);
  w->gm.sn = take((long long)b * steps);
  w->gm.g = take((long long)b * (steps + 1));
  w->gm.beta = take(b);
  w->gm.scale = take(b);
  w->gm.y = take((long long)b * steps);
  w->gm.h = take((long long)b * (steps + 1));
  w->gm.nrm2 = take(b);
  w->keep = reinterpret_cast<int *>(take(bw));
  w->keep0 = reinterpret_cast<int *>(take(bw));
  w->gstate = reinterpret_cast<int *>(take(2));
  w->gshift = take(1);
  w->jstat = reinterpret_cast<int *>(take(4));  // 8 counters
  w->dgks = reinterpret_cast<int *>(take(2));
  w->gm.done = reinterpret_cast<int *>(take(b));
  w->gm.mvalid = reinterpret_cast<int *>(take(b));
  if ((char *)p > (char *)w->arena + bytes) return set_error(ctx, TPS_ERR_CUDA, "arena overflow");
  TPS_CUDA_TRY(ctx, cudaMemset(w->arena, 0, bytes));
  // the memset runs on the legacy default stream; the solve's stream may be non-blocking
  TPS_CUDA_TRY(ctx, cudaStreamSynchronize(cudaStreamLegacy));
  TPS_CUDA_TRY(ctx, cudaMallocHost((void **)&w->h_pinned, 4096 * sizeof(double)));
  TPS_CUDA_TRY(ctx, cudaMallocHost((void **)&w->hi_pinned, 4096 * sizeof(int)));
  // the Gram scratch must hold the largest skinny product of the loop
  int st = ensure_gram_scratch(ctx, gram_scratch_doubles(std::max(q, mmax), std::max(q, mmax), 1));
  if (st) return st;
  // preconditioner intermediates for a block of b vectors
  return ensure_apply_workspace(ctx, (long long)std::max(b, q) * N);
}

}  // namespace

void free_solver_workspace(tps_ctx *ctx) {
  if (!ctx->sw) return;
  ctx->sw->tm.destroy();
  if (ctx->sw->capture) cudaStreamDestroy(ctx->sw->capture);
  cudaFree(ctx->sw->arena);
  cudaFreeHost(ctx->sw->h_pinned);
  cudaFreeHost(ctx->sw->hi_pinned);
  delete ctx->sw;
  ctx->sw = nullptr;
}

// GMRES on the projected, preconditioned correction equation for nsys systems in
// lockstep (Eq. jdcor; Sec. 4.1: GMRES with the preconditioner of Sec. 4.2).  Qt: nq
// orthonormal columns; KQt: K^-1 Qt if already computed (nq_cached of the columns; the
// rest are computed here), theta: device [nsys].  Writes T [nsys][N].
int correction_impl(tps_ctx *ctx, const DevOperator &op, const double *Qt, int nq,
                    const double *KQt_cached, int nq_cached, const double *R,
                    const double *theta, int nsys, int steps, int use_prec, double shift,
                    double inner_tol, double *T, int *h_applies, int *prec_applies,
                    cudaStream_t s, bool direction_only, bool low, const double *shift_dev) {
  SolverWorkspace &w = *ctx->sw;
  Ctx c{ctx, op, w, s, op.N};
  const long long N = op.N;
  double *KQt = w.KQX;
  if (use_prec && nq > 0) {
    if (KQt_cached != KQt && nq_cached > 0)
      TPS_CUDA_TRY(ctx, cudaMemcpyAsync(KQt, KQt_cached, (size_t)nq_cached * N * sizeof(double),
                                        cudaMemcpyDeviceToDevice, s));
    if (nq > nq_cached) {
      apply_prec_timed(c, Qt + (long long)nq_cached * N, KQt + (long long)nq_cached * N,
                       nq - nq_cached, shift, shift_dev);
      *prec_applies += nq - nq_cached;
    }
    tgram(Qt, N, 0, nq, KQt, N, 0, nq, N, w.Mq, nq, 0, 1, ctx->gscr, s, nullptr, w.corr_low);
    launch_spd_inverse(w.Mq, nq, w.Minv, s);
  }
  const int sst = steps;
  // z_0 = -Kt^-1 r / beta
  double *Z = w.Z;
  kt_inverse(c, Qt, nq, KQt, use_prec, shift, R, nsys, Z, shift_dev);
  if (use_prec) *prec_applies += nsys;
  if (direction_only && sst == 1) {
    // one GMRES step only scales z_0, and the caller normalises the correction: the
    // correction direction is the projected, preconditioned residual -Kt^-1 r
    launch_axpby_cols(nsys, N, -1.0, Z, N, 0.0, T, N, s);
    TPS_CUDA_TRY(ctx, cudaGetLastError());
    return TPS_OK;
  }
  col_norms2(c, Z, nsys, w.gm.nrm2);
  launch_gmres_init(nsys, sst, w.gm.nrm2, w.gm, s);
  launch_scale_cols(nsys, N, Z, N, w.gm.scale, 0, Z, N, s);
  for (int j = 0; j < sst; ++j) {
    double *zj = Z + (long long)j * nsys * N;
    // right projector of Eq. jdcor, applied explicitly: rounding in the Q directions
    // would otherwise grow by 1/h_{j+1,j} per Arnoldi step
    if (nq > 0) {
      tgram(Qt, N, 0, nq, zj, N, 0, nsys, N, w.C, nq, 0, 1, ctx->gscr, s, nullptr, w.corr_low);
      tupdate(Qt, N, 0, nq, w.C, nq, 0, nsys, -1.0, 1.0, zj, N, 0, N, 1, s, nullptr, w.corr_low);
    }
    apply_h_timed(c, zj, w.W, nsys, theta, low);
    *h_applies += nsys;
    kt_inverse(c, Qt, nq, KQt, use_prec, shift, w.W, nsys, w.P, shift_dev);
    if (use_prec) *prec_applies += nsys;
    // Arnoldi, classical Gram-Schmidt twice, per system: h = Z_i^T p_i ; p_i -= Z_i h
    for (int pass = 0; pass < 2; ++pass) {
      tgram(Z, (long long)nsys * N, N, j + 1, w.P, N, N, 1, N, w.gm.h, sst + 1, sst + 1, nsys,
            ctx->gscr, s, nullptr, w.corr_low);
      tupdate(Z, (long long)nsys * N, N, j + 1, w.gm.h, sst + 1, sst + 1, 1, -1.0, 1.0, w.P, N,
              N, N, nsys, s, nullptr, w.corr_low);
      launch_hess_add(nsys, sst, j, w.gm.h, sst + 1, w.gm, s);
    }
    col_norms2(c, w.P, nsys, w.gm.nrm2);
    launch_gmres_givens(nsys, sst, j, w.gm.nrm2, w.gm, inner_tol, s);
    launch_scale_cols(nsys, N, w.P, N, w.gm.scale, 0, Z + (long long)(j + 1) * nsys * N, N, s);
  }
  launch_gmres_solve(nsys, sst, w.gm, s);
  tupdate(Z, (long long)nsys * N, N, sst, w.gm.y, sst, sst, 1, 1.0, 0.0, T, N, N, N, nsys, s,
          nullptr, w.corr_low);
  TPS_CUDA_TRY(ctx, cudaGetLastError());
  return TPS_OK;
}

int solve_impl(tps_ctx *ctx, int k, int parity, double tol, int block, const double *x0,
               int n_x0, const tps_solver_opts *opts_in, double *evals_host, double *evecs_dev,
               tps_stats *stats, cudaStream_t s) {
  const auto t_start = std::chrono::steady_clock::now();
  tps_solver_opts opts;
  tps_default_opts(&opts);
  if (opts_in) opts = *opts_in;
  const int k_req = k;
  k = k_req + std::max(0, opts.guard);  // converge k + guard pairs, return the lowest k
  const int b = std::min(block, k);
  int mmin = opts.m_min > 0 ? opts.m_min : std::max(2 * k, 8);
  mmin = ((mmin + b - 1) / b) * b;
  int mmax = opts.m_max > 0 ? opts.m_max : mmin + 2 * b;
  mmax = std::min(mmax, 64);
  if (mmin > mmax - b) mmin = std::max(b, mmax - b);
  if (mmin < k) mmin = std::min(k, mmax - b);
  // GMRES steps per correction: fixed when given, else adaptive -- start with one step
  // (the projected preconditioned residual) and widen when the outer residual stalls
  const bool adaptive_steps = opts.inner_steps <= 0;
  const int steps_max = adaptive_steps ? 10 : opts.inner_steps;
  int steps = adaptive_steps ? 1 : opts.inner_steps;
  const int max_outer = opts.max_outer > 0 ? opts.max_outer : 500;
  const double inner_tol = opts.inner_tol > 0 ? opts.inner_tol : 1e-3;
  const bool mixed = opts.h_dtype == TPS_F32;
  // refinement phase block (default: all k + guard pairs at once) and search space
  const int rb = std::min(32, std::min(k, opts.refine_block > 0 ? opts.refine_block : k));
  int rmmin = ((std::max(2 * k, 8) + rb - 1) / rb) * rb;
  int rmmax = std::min(64, rmmin + 2 * rb);
  if (rmmin > rmmax - rb) rmmin = std::max(rb, rmmax - rb);
  const double switch_tol = opts.switch_tol > 0 ? std::max(opts.switch_tol, tol) : std::max(1e-6, tol);
  if (mmax < 2 * b || steps_max > 40)
    return set_error(ctx, TPS_ERR_INVALID_ARG, "search space too small for the block");

  const DevOperator *opp = &ctx->full;
  if (parity != TPS_ANY) {
    int st = build_sector_operator(ctx, parity);
    if (st) return st;
    opp = &ctx->sect[parity];
  }
  const DevOperator &op = *opp;
  const long long N = op.N;
  if (k_req > N / 2) return set_error(ctx, TPS_ERR_INVALID_ARG, "k too large for the grid");
  if (k > N / 2) k = (int)(N / 2);
  int st = alloc_workspace(ctx, N, std::max(mmax, rmmax), std::max(b, rb), k,
                           std::max(steps_max, opts.refine_inner_steps));
  if (st) return st;
  SolverWorkspace &w = *ctx->sw;
  Ctx c{ctx, op, w, s, N};
  w.tm.reset(opts.timing != 0);
  TPS_CUDA_TRY(ctx, cudaMemsetAsync(w.jstat, 0, 8 * sizeof(int), s));
  TPS_CUDA_TRY(ctx, cudaMemsetAsync(w.dgks, 0, 4 * sizeof(int), s));
  // per-solve thread-local state of tupdate/tgram: the phase timers and the update arithmetic
  struct SolveScope {
    explicit SolveScope(PhaseTiming *t, bool split, bool split_gram) {
      tl_timing = t;
      tl_split_updates = split;
      tl_split_grams = split_gram;
    }
    ~SolveScope() {
      tl_timing = nullptr;
      tl_split_updates = false;
      tl_split_grams = false;
    }
  } solve_scope(&w.tm, opts.update_dtype == TPS_F64_TC, opts.gram_dtype == TPS_F64_TC);
  // the TF32 tensor-core preconditioner: 1D, and 2D grids whose modes it takes (else FP32)
  w.prec_dtype = opts.prec_dtype == TPS_F64
                     ? TPS_F64
                     : ((opts.prec_dtype == TPS_TF32_TC && tf_prec_supported(op)) ? TPS_TF32_TC
                                                                                 : TPS_F32);
  w.corr_low = opts.correction_dtype != TPS_F64;
  if (w.prec_dtype == TPS_TF32_TC) {
    const int st_tf = ensure_tf_operator(op);  // allocation errors here, not mid-solve
    if (st_tf) return set_error(ctx, st_tf, "building the TF32 preconditioner operator failed");
  }
  // the tensor-core FP64 H-apply: 1D, and 2D with at most 128 points per mode (else the
  // FMA pipe)
  bool tc_ok = op.nmodes == 2;
  if (op.nmodes == 4) {
    tc_ok = true;
    for (int kk = 0; kk < 4; ++kk) tc_ok = tc_ok && op.n[kk] <= 128;
  }
  w.h64_dtype = (opts.h64_dtype == TPS_F64_TC && tc_ok) ? TPS_F64_TC : TPS_F64;
  if (w.h64_dtype == TPS_F64_TC)
    TPS_CUDA_TRY(ctx, ensure_tc_operator(op, s));  // allocation errors here, not mid-solve
  const long long launches0 = g_kernel_launches.load();
  double hnorm = 0.0;
  tps_get_info(ctx, nullptr, &hnorm);

  tps_stats stt;
  std::memset(&stt, 0, sizeof(stt));
  stt.hnorm_est = hnorm;
  uint64_t rng_counter = 0;
  std::vector<double> lam(k, 0.0), resid(k, 0.0);

  // start block: warm start restricted to the sector, completed with random columns.  A
  // warm start may fill a first block as wide as all k + guard wanted pairs: a start that
  // holds only the first b of them leaves the rest to be found late (the corrections aim
  // at the states already present)
  int bn = b;
  {
    const int nw = std::min(n_x0, std::max(b, k));
    if (nw > b) bn = nw;
    if (nw > 0 && x0) {
      if (parity != TPS_ANY)
        launch_sector_restrict(parity, ctx->n[0], ctx->n[1], nw, x0, w.V, s);
      else
        TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.V, x0, (size_t)nw * N * sizeof(double),
                                          cudaMemcpyDeviceToDevice, s));
    }
    if (nw < b) {
      double *Rb = w.V + (long long)nw * N;
      st = fill_random(c, Rb, b - nw, opts.seed, rng_counter);
      if (st) return st;
      // low-pass filter the random columns: (T - s)^-1 applied smooth_start times
      const double s_smooth = op.lam_min_sum - 1e-3 * hnorm;
      for (int it = 0; it < opts.smooth_start && opts.use_prec; ++it) {
        apply_prec_timed(c, Rb, w.P, b - nw, s_smooth);
        TPS_CUDA_TRY(ctx, cudaMemcpyAsync(Rb, w.P, (size_t)(b - nw) * N * sizeof(double),
                                          cudaMemcpyDeviceToDevice, s));
        stt.prec_applies += b - nw;
      }
    }
  }
  // one phase of the outer loop: starts from the bn columns in V, locks pairs whose
  // residual reaches tol_p * ||H||_est into QX; low = true runs the H-applies in FP32
  int m = 0, nlock = 0, outer = 0, bn_phase = bn;
  bool converged = false;
  // bp/mminp/mmaxp: block and search-space sizes of the phase; inner_low: FP32 H inside
  // the GMRES correction solves
  // G and Y are stored with the allocated search-space size as leading dimension, which
  // covers every phase's m_max
  const int ldG = w.mmax;
  auto run_phase = [&](bool low, double tol_p, int bn0, int bp, int mminp, int mmaxp,
                       bool fixed_steps, int steps_p, bool inner_low) -> int {
  if (fixed_steps) steps = steps_p;
  m = 0;
  nlock = 0;
  converged = false;
  int bn = bn0;
  double cached_shift = NAN;
  int kq_valid = 0;  // locked columns of KQX valid for cached_shift
  double prev_res = INFINITY;
  int stall = 0, prev_nlock = -1;
  int warm_mp = 0;  // leading block of G already diagonalised by the last Jacobi call
  // Ritz vectors are only needed to a fraction of the current residuals: the Jacobi
  // eigensolve stops at 1e-3 of the smallest unconverged residual of the last iteration
  // (its exact result Y^T G Y is kept in Arot, so no inexactness accumulates in G)
  double jac_tol = 0.0;
  int st = TPS_OK;
  for (; outer < max_outer; ++outer) {
    // (1) orthonormalise the new block against the locked vectors and the basis
    double *T = w.V + (long long)m * N;
    int rank = 0;
    for (int attempt = 0; attempt < 3; ++attempt) {
      st = orthonormalize(c, w.QX, nlock, w.V, m, T, bn, &rank);
      if (st) return st;
      if (rank > 0) break;
      st = fill_random(c, T, bn, opts.seed, rng_counter);
      if (st) return st;
    }
    if (rank == 0) return set_error(ctx, TPS_ERR_NOT_CONVERGED, "search space cannot be expanded");
    bn = rank;
    // (2) H applied to the new block
    double *HT = w.HV + (long long)m * N;
    apply_h_timed(c, T, HT, bn, nullptr, low);
    stt.h_applies += bn;
    // (3) projected matrix G = V^T H V, new columns and their mirror
    if (m > 0) tgram(w.V, N, 0, m, HT, N, 0, bn, N, w.G + (long long)m * ldG, ldG, 0, 1,
                           ctx->gscr, s);
    tgram(T, N, 0, bn, HT, N, 0, bn, N, w.G + (long long)m * ldG + m, ldG, 0, 1, ctx->gscr,
                s);
    launch_mirror_block(w.G, ldG, m, bn, s);
    m += bn;
    // (4) Rayleigh-Ritz
    {
      PhaseTiming &t = w.tm;
      const bool rec = t.on && (t.seen[5]++ % PhaseTiming::kSample) == 0;
      cudaEvent_t ea = nullptr, eb = nullptr;
      if (rec) {
        ea = t.get();
        eb = t.get();
        cudaEventRecord(ea, s);
      }
      launch_rr_eigh(w.G, m, ldG, w.theta, w.Y, ldG, s, warm_mp, w.jstat, jac_tol, w.Arot,
                     opts.rr_method, opts.rr_refine_max);
      t.launches[5] += 1;
      if (rec) {
        cudaEventRecord(eb, s);
        t.pend[5].push_back({ea, eb});
        t.timed[5] += 1;
      }
    }
    warm_mp = m;  // valid for the next iteration unless the basis is rotated below
    const int nact = std::min(bp, std::min(k - nlock, m));
    double *X = w.QX + (long long)nlock * N;
    tupdate(w.V, N, 0, m, w.Y, ldG, 0, nact, 1.0, 0.0, X, N, 0, N, 1, s);
    tupdate(w.HV, N, 0, m, w.Y, ldG, 0, nact, 1.0, 0.0, w.HX, N, 0, N, 1, s);
    launch_residual(nact, N, w.HX, X, w.theta, w.R, s);
    col_norms2(c, w.R, nact, w.nrm2);
    // (5) read back Ritz values and residual norms
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.h_pinned, w.theta, nact * sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.h_pinned + 64, w.nrm2, nact * sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
    TPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    TPS_CUDA_TRY(ctx, cudaGetLastError());
    w.tm.drain();
    int nconv = 0;
    while (nconv < nact && std::sqrt(std::max(w.h_pinned[64 + nconv], 0.0)) <= tol_p * hnorm) {
      lam[nlock + nconv] = w.h_pinned[nconv];
      resid[nlock + nconv] = std::sqrt(std::max(w.h_pinned[64 + nconv], 0.0)) / hnorm;
      ++nconv;
    }
    if (!std::isfinite(w.h_pinned[0]))
      return set_error(ctx, TPS_ERR_NOT_CONVERGED, "non-finite Ritz value");
    {
      double rmin = INFINITY;
      for (int i = nconv; i < nact; ++i)
        rmin = std::min(rmin, std::sqrt(std::max(w.h_pinned[64 + i], 0.0)));
      jac_tol = std::isfinite(rmin) ? 1e-3 * rmin : 0.0;
    }
    nlock += nconv;
    if (nlock >= k) {
      converged = true;
      ++outer;
      break;
    }
    if (adaptive_steps && !fixed_steps && nconv < nact) {
      // stall detection on the lowest unconverged pair: two outer iterations in a row
      // without halving its residual widen the inner solve
      const double res0 = std::sqrt(std::max(w.h_pinned[64 + nconv], 0.0));
      if (nlock != prev_nlock) {
        prev_nlock = nlock;
        stall = 0;
      } else {
        stall = (res0 > 0.5 * prev_res) ? stall + 1 : 0;
      }
      prev_res = res0;
      if (stall >= 2 && steps < steps_max) {
        steps = std::min(2 * steps + 1, steps_max);
        stall = 0;
      }
    }
    // (6) lock and/or restart: keep Ritz vectors nconv .. nconv+mk-1
    int nact2 = nact;
    if (nconv > 0 || m + bp > mmaxp) {
      const int avail = m - nconv;
      const int mk = (m + bp > mmaxp) ? std::min(avail, mminp) : avail;
      // Ritz vectors nconv .. nact-1 are already in X and HX (columns nconv .. of the
      // block formed for the residuals, by the same products in the same order): copy
      // them, and form only the remaining kept columns
      const int ov = std::max(0, std::min(nact - nconv, mk));
      if (ov > 0) {
        TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.V2, X + (long long)nconv * N,
                                          (size_t)ov * N * sizeof(double),
                                          cudaMemcpyDeviceToDevice, s));
        TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.HV2, w.HX + (long long)nconv * N,
                                          (size_t)ov * N * sizeof(double),
                                          cudaMemcpyDeviceToDevice, s));
      }
      if (mk > ov) {
        tupdate(w.V, N, 0, m, w.Y + (long long)(nconv + ov) * ldG, ldG, 0, mk - ov, 1.0, 0.0,
                w.V2 + (long long)ov * N, N, 0, N, 1, s);
        tupdate(w.HV, N, 0, m, w.Y + (long long)(nconv + ov) * ldG, ldG, 0, mk - ov, 1.0, 0.0,
                w.HV2 + (long long)ov * N, N, 0, N, 1, s);
      }
      std::swap(w.V, w.V2);
      std::swap(w.HV, w.HV2);
      launch_copy_small(w.theta + nconv, w.theta2, mk, s);
      std::swap(w.theta, w.theta2);
      launch_copy_block(w.Arot, ldG, nconv, w.G, ldG, mk, s);  // G in the kept Ritz basis
      m = mk;
      warm_mp = 0;  // G's leading block is diagonal by construction
      ++stt.restarts;
      nact2 = std::min(bp, std::min(k - nlock, m));
      X = w.QX + (long long)nlock * N;
      TPS_CUDA_TRY(ctx, cudaMemcpyAsync(X, w.V, (size_t)nact2 * N * sizeof(double),
                                        cudaMemcpyDeviceToDevice, s));
      TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.HX, w.HV, (size_t)nact2 * N * sizeof(double),
                                        cudaMemcpyDeviceToDevice, s));
      launch_residual(nact2, N, w.HX, X, w.theta, w.R, s);
    }
    // (7) correction equations for the active Ritz pairs
    // Preconditioner shift.  The kinetic part T is positive semi-definite with its
    // bottom at lam_min_sum (= 0), so K = T - shift is positive definite for any
    // shift below it.  The paper's choice is the two-body threshold -E0 (Sec. 4.2),
    // just above the wanted bound states; without E0 the adaptive choice is the
    // lowest active Ritz value when it lies below the kinetic spectrum, else its
    // mirror image below it (a positive shift would make K indefinite).
    double shift = opts.prec_shift;
    if (!std::isfinite(shift)) {
      const double th0 = w.h_pinned[nconv < nact ? nconv : 0];
      const double floor_gap = std::max(std::fabs(th0 - op.lam_min_sum), 1e-8 * hnorm);
      shift = op.lam_min_sum - floor_gap;
    }
    // keep the previous shift (and the cached K^-1 of the locked vectors) while the
    // adaptive choice moves by less than 10 %: the preconditioner only approximates
    // (H - theta)^-1, so a slightly older shift costs nothing in convergence
    if (!std::isfinite(opts.prec_shift) && std::isfinite(cached_shift) &&
        std::fabs(shift - cached_shift) <= 0.1 * std::fabs(cached_shift))
      shift = cached_shift;
    if (opts.use_prec && !(shift == cached_shift)) {
      kq_valid = 0;
      cached_shift = shift;
    }
    const int nq = nlock + nact2;
    // K^-1 of newly locked columns is recomputed each time (kq_valid tracks the cache)
    st = correction_impl(ctx, op, w.QX, nq, w.KQX, opts.use_prec ? std::min(kq_valid, nlock) : 0,
                         w.R, w.theta, nact2, steps, opts.use_prec, shift, inner_tol,
                         w.V + (long long)m * N, &stt.h_applies, &stt.prec_applies, s, true,
                         low || inner_low);
    if (st) return st;
    kq_valid = nlock;
    stt.inner_steps += steps * nact2;
    bn = nact2;
  }
  return TPS_OK;
  };
  if (!mixed) {
    st = run_phase(false, tol, bn_phase, b, mmin, mmax, false, 0, false);
    if (st) return st;
  } else {
    // low-precision phase: FP32 mode products until every pair reaches switch_tol, then
    // an FP64 refinement from that subspace, all pairs in the first block
    st = run_phase(true, switch_tol, bn_phase, b, mmin, mmax, false, 0, false);
    if (st) return st;
    if (converged) {
      const int nk = std::min(nlock, k);
      TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.V, w.QX, (size_t)nk * N * sizeof(double),
                                        cudaMemcpyDeviceToDevice, s));
      stt.restarts += 1;
      st = run_phase(false, tol, nk, rb, rmmin, rmmax, opts.refine_inner_steps > 0,
                     opts.refine_inner_steps, opts.refine_inner_dtype == TPS_F32);
      if (st) return st;
    }
  }
  stt.outer_iters = outer;
  // final Rayleigh quotients and residuals with a fresh H-apply of the locked vectors
  const int nlocked = std::min(nlock, k);
  int nret = 0;
  if (nlocked > 0) {
    const int nl = nlocked;
    double *HQ = w.V2;  // at least max(mmax, kmax) columns
    apply_h_timed(c, w.QX, HQ, nl, nullptr, false);
    stt.h_applies += nl;
    tgram(w.QX, N, N, 1, HQ, N, N, 1, N, w.theta2, 1, 1, nl, ctx->gscr, s);
    col_norms2(c, w.QX, nl, w.ref);
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.h_pinned, w.theta2, nl * sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.h_pinned + 1024, w.ref, nl * sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
    TPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    for (int i = 0; i < nl; ++i) lam[i] = w.h_pinned[i] / w.h_pinned[1024 + i];
    // final residual norms ||H x - lambda x|| / ||H||_est
    for (int i = 0; i < nl; ++i) w.h_pinned[2048 + i] = lam[i];
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.theta2, w.h_pinned + 2048, nl * sizeof(double),
                                      cudaMemcpyHostToDevice, s));
    launch_residual(nl, N, HQ, w.QX, w.theta2, w.HV2, s);
    col_norms2(c, w.HV2, nl, w.ref);
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.h_pinned + 3072, w.ref, nl * sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
    TPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    for (int i = 0; i < nl; ++i) resid[i] = std::sqrt(std::max(w.h_pinned[3072 + i], 0.0)) / hnorm;
    // sort ascending (locking order is ascending up to rounding within clusters)
    std::vector<int> order(nl);
    for (int i = 0; i < nl; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int bb) { return lam[a] < lam[bb]; });
    // expand the lowest k_req to the full grid in sorted order
    nret = std::min(nl, k_req);
    for (int i = 0; i < nret; ++i) {
      const double *src = w.QX + (long long)order[i] * N;
      double *dst = evecs_dev + (long long)i * ctx->full.N;
      if (parity != TPS_ANY)
        launch_sector_expand(parity, ctx->n[0], ctx->n[1], 1, src, dst, s);
      else
        TPS_CUDA_TRY(ctx, cudaMemcpyAsync(dst, src, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      evals_host[i] = lam[order[i]];
      if (i < 64) stt.resid[i] = resid[order[i]];
    }
    launch_fix_sign(nret, ctx->full.N, evecs_dev, ctx->gscr, s);
    TPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    TPS_CUDA_TRY(ctx, cudaGetLastError());
  }
  w.tm.drain();
  stt.n_converged = nret;
  stt.h_ms = w.tm.ms[0];
  stt.prec_ms = w.tm.ms[1];
  stt.h_flops = w.tm.flops[0];
  stt.prec_flops = w.tm.flops[1];
  stt.h_launches = w.tm.launches[0];
  stt.prec_launches = w.tm.launches[1];
  stt.h32_ms = w.tm.ms[2];
  stt.h32_flops = w.tm.flops[2];
  stt.h32_launches = w.tm.launches[2];
  {
    int js[8] = {0, 0, 0, 0, 0, 0, 0, 0}, gs[4] = {0, 0, 0, 0};
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.hi_pinned + 2048, w.jstat, 8 * sizeof(int),
                                      cudaMemcpyDeviceToHost, s));
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.hi_pinned + 2056, w.dgks, 3 * sizeof(int),
                                      cudaMemcpyDeviceToHost, s));
    TPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    std::memcpy(js, w.hi_pinned + 2048, 8 * sizeof(int));
    std::memcpy(gs, w.hi_pinned + 2056, 3 * sizeof(int));
    stt.gs_second_passes = gs[1];
    stt.gs_orthogonalisations = gs[2];
    stt.jacobi_sweeps = js[0];
    stt.jacobi_rounds = js[1];
    stt.jacobi_calls = js[2];
    stt.rr_mixed_calls = js[3];
    stt.rr_fp32_solves = js[4];
    stt.rr_refine_iters = js[5];
    stt.rr_groups_rotated = js[6];
    stt.rr_fallbacks = js[7];
  }
  stt.gram_ms = w.tm.ms[3];
  stt.gram_flops = w.tm.flops[3];
  stt.gram_bytes = w.tm.bytes[3];
  stt.gram_launches = w.tm.launches[3];
  stt.upd_ms = w.tm.ms[4];
  stt.upd_flops = w.tm.flops[4];
  stt.upd_bytes = w.tm.bytes[4];
  stt.upd_launches = w.tm.launches[4];
  stt.rr_ms = w.tm.ms[5];
  stt.rr_launches = w.tm.launches[5];
  stt.rr_timed = w.tm.timed[5];
  stt.kernel_launches = g_kernel_launches.load() - launches0;
  stt.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (stats) *stats = stt;
  {
    TPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    const int f = (w.h64_dtype == TPS_F64_TC ? tc_operator_status(op) : 0) |
                  (opts.update_dtype == TPS_F64_TC ? update_split_status() : 0);
    if (f < 0) return set_error(ctx, TPS_ERR_CUDA, "reading the device status flag failed");
    if (f) return set_error(ctx, TPS_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait");
  }
  if (!converged) return set_error(ctx, TPS_ERR_NOT_CONVERGED, "outer-iteration cap reached");
  return TPS_OK;
}

// ---------------------------------------------------------------------------------------
// The outer loop as a captured CUDA graph (tps_solver_opts.graph).  With every wanted pair
// in one block (b = k), no locking, the preconditioner shift kept on the device (a kernel
// sets it from the lowest unconverged Ritz value each iteration, unless prec_shift fixes it)
// and one preconditioned-residual step per correction (the projected direction -Kt^-1 r of
// Eq. jdcor), the search space follows a fixed cycle -- m = m_min -> m_min + b -> m_max =
// m_min + 2b, restart to m_min -- and every kernel of an outer iteration has sizes known in
// advance.  The only data-dependent decision, "converged?", is taken on the device
// (k_conv_check) and drives a conditional WHILE node around the captured two-iteration
// cycle, so after the eager iterations that fill the first m_min columns (the last of them
// fixes the shift from the lowest Ritz value) the rest of the solve is one graph launch
// with no host round trip.  Columns that the orthonormalisation drops
// become zero and get a diagonal in G above the wanted Ritz values instead of being
// compacted on the host.
namespace {

struct GraphIter {
  int m;          // search-space size before the expansion
  bool restart;   // restart to 2b after this iteration
};

// One outer iteration with static sizes: orthonormalise the block at V + m, apply H, extend
// G, Ritz pairs, targets X/HX/R and their residual norms, optional restart, correction of
// all b targets into the next block.  Returns the search-space size after it.
int graph_iteration(Ctx &c, const GraphIter &it, int b, int mmin, double shift, bool use_prec,
                    int *h_applies, int *prec_applies, double thresh2, double hnorm,
                    bool dev_shift) {
  SolverWorkspace &w = c.w;
  const long long N = c.N;
  const int m = it.m, ldG = w.mmax;
  double *T = w.V + (long long)m * N;
  // block CGS2 (second pass only where the first lost more than half a column's norm) and
  // Cholesky-QR twice; dropped columns stay as zeros (keep0)
  col_norms2(c, T, b, w.ref);
  for (int pass = 0; pass < 2 && m > 0; ++pass) {
    const int *need = nullptr;
    if (pass == 1) {
      col_norms2(c, T, b, w.nrm2);
      launch_dgks_flag(w.ref, w.nrm2, b, w.dgks, w.dgks + 1, c.s);
      need = w.dgks;
    }
    tgram(w.V, N, 0, m, T, N, 0, b, N, w.C, m, 0, 1, c.ctx->gscr, c.s, need);
    tupdate(w.V, N, 0, m, w.C, m, 0, b, -1.0, 1.0, T, N, 0, N, 1, c.s, need);
  }
  for (int pass = 0; pass < 2; ++pass) {
    tgram(T, N, 0, b, T, N, 0, b, N, w.C, b, 0, 1, c.ctx->gscr, c.s);
    launch_chol_inv(w.C, b, pass == 0 ? w.ref : nullptr, pass == 0 ? 1e-7 : 1e-12, w.Rinv,
                    w.keep, c.s);
    tupdate(T, N, 0, b, w.Rinv, b, 0, b, 1.0, 0.0, w.T2, N, 0, N, 1, c.s, nullptr, false, false);
    cudaMemcpyAsync(T, w.T2, (size_t)b * N * sizeof(double), cudaMemcpyDeviceToDevice, c.s);
    if (pass == 0) cudaMemcpyAsync(w.keep0, w.keep, b * sizeof(int), cudaMemcpyDeviceToDevice, c.s);
  }
  double *HT = w.HV + (long long)m * N;
  apply_h_timed(c, T, HT, b, nullptr, false);
  *h_applies += b;
  if (m > 0) tgram(w.V, N, 0, m, HT, N, 0, b, N, w.G + (long long)m * ldG, ldG, 0, 1, c.ctx->gscr, c.s);
  tgram(T, N, 0, b, HT, N, 0, b, N, w.G + (long long)m * ldG + m, ldG, 0, 1, c.ctx->gscr, c.s);
  launch_mirror_block(w.G, ldG, m, b, c.s);
  launch_mark_dropped(w.G, ldG, m, b, w.keep0, c.s);
  const int mm = m + b;
  launch_rr_eigh(w.G, mm, ldG, w.theta, w.Y, ldG, c.s, 0, w.jstat, 0.0, w.Arot, TPS_RR_MIXED, 0);
  tupdate(w.V, N, 0, mm, w.Y, ldG, 0, b, 1.0, 0.0, w.QX, N, 0, N, 1, c.s);
  tupdate(w.HV, N, 0, mm, w.Y, ldG, 0, b, 1.0, 0.0, w.HX, N, 0, N, 1, c.s);
  launch_residual(b, N, w.HX, w.QX, w.theta, w.R, c.s);
  col_norms2(c, w.R, b, w.nrm2);
  // converged pairs get no correction; the shift follows the lowest unconverged Ritz value
  launch_zero_converged(w.R, N, w.nrm2, b, thresh2, c.s);
  if (dev_shift)
    launch_shift_update(w.theta, w.nrm2, b, thresh2, c.op.lam_min_sum, hnorm, w.gshift, c.s);
  int mnew = mm;
  if (it.restart) {  // keep the lowest mmin Ritz vectors (theta[0 .. mmin) stay in place)
    tupdate(w.V, N, 0, mm, w.Y, ldG, 0, mmin, 1.0, 0.0, w.V2, N, 0, N, 1, c.s);
    tupdate(w.HV, N, 0, mm, w.Y, ldG, 0, mmin, 1.0, 0.0, w.HV2, N, 0, N, 1, c.s);
    cudaMemcpyAsync(w.V, w.V2, (size_t)mmin * N * sizeof(double), cudaMemcpyDeviceToDevice, c.s);
    cudaMemcpyAsync(w.HV, w.HV2, (size_t)mmin * N * sizeof(double), cudaMemcpyDeviceToDevice, c.s);
    launch_copy_block(w.Arot, ldG, 0, w.G, ldG, mmin, c.s);  // G in the kept Ritz basis
    mnew = mmin;
  }
  correction_impl(c.ctx, c.op, w.QX, b, nullptr, 0, w.R, w.theta, b, 1, use_prec ? 1 : 0, shift,
                  1e-3, w.V + (long long)mnew * N, h_applies, prec_applies, c.s, true, w.corr_low,
                  dev_shift ? w.gshift : nullptr);
  return mnew;
}

}  // namespace

int solve_graph_impl(tps_ctx *ctx, int k_req, int parity, double tol,
                     const tps_solver_opts &opts, double *evals_host, double *evecs_dev,
                     tps_stats *stats, cudaStream_t s) {
  const auto t_start = std::chrono::steady_clock::now();
  // every wanted pair in the one block; the Rayleigh-Ritz space (up to 6 k) plays the role
  // of the guard pairs
  const int k = k_req;
  const int b = k;
  // default m_min = 4k (measured on the 256-instance sweep: 12, 16, 20, 24 at k = 4 took
  // 34, 28, 26, 24 outer iterations, 16 the least time), at most 64 - 2k
  const int m0 = opts.m_min > 0 ? opts.m_min : std::max(4 * k, 8);
  int mmin = ((m0 + b - 1) / b) * b;
  if (mmin + 2 * b > 64) mmin = ((64 - 2 * b) / b) * b;
  const int mmax = mmin + 2 * b;
  if (b > 16 || mmin < b) return set_error(ctx, TPS_ERR_INVALID_ARG, "graph solver: k <= 16");
  const DevOperator *opp = &ctx->full;
  if (parity != TPS_ANY) {
    int st = build_sector_operator(ctx, parity);
    if (st) return st;
    opp = &ctx->sect[parity];
  }
  const DevOperator &op = *opp;
  const long long N = op.N;
  if (k > N / 2) return set_error(ctx, TPS_ERR_INVALID_ARG, "k too large for the grid");
  int st = alloc_workspace(ctx, N, mmax, b, k, 1);
  if (st) return st;
  SolverWorkspace &w = *ctx->sw;
  Ctx c{ctx, op, w, s, N};
  w.tm.reset(false);
  w.prec_dtype = opts.prec_dtype == TPS_F64 ? TPS_F64
                 : (opts.prec_dtype == TPS_TF32_TC && tf_prec_supported(op)) ? TPS_TF32_TC
                                                                             : TPS_F32;
  w.corr_low = opts.correction_dtype != TPS_F64;
  w.h64_dtype = (opts.h64_dtype == TPS_F64_TC && op.nmodes == 2) ? TPS_F64_TC : TPS_F64;
  if (w.prec_dtype == TPS_TF32_TC) {
    const int st_tf = ensure_tf_operator(op);
    if (st_tf) return set_error(ctx, st_tf, "building the TF32 preconditioner operator failed");
  }
  if (w.h64_dtype == TPS_F64_TC) TPS_CUDA_TRY(ctx, ensure_tc_operator(op, s));
  struct Scope {
    explicit Scope(bool split, bool split_gram) {
      tl_timing = nullptr;
      tl_split_updates = split;
      tl_split_grams = split_gram;
    }
    ~Scope() {
      tl_split_updates = false;
      tl_split_grams = false;
    }
  } scope(opts.update_dtype == TPS_F64_TC, opts.gram_dtype == TPS_F64_TC);
  const long long launches0 = g_kernel_launches.load();
  double hnorm = 0.0;
  tps_get_info(ctx, nullptr, &hnorm);
  tps_stats stt;
  std::memset(&stt, 0, sizeof(stt));
  stt.hnorm_est = hnorm;
  TPS_CUDA_TRY(ctx, cudaMemsetAsync(w.jstat, 0, 8 * sizeof(int), s));
  TPS_CUDA_TRY(ctx, cudaMemsetAsync(w.dgks, 0, 4 * sizeof(int), s));
  TPS_CUDA_TRY(ctx, cudaMemsetAsync(w.gstate, 0, 2 * sizeof(int), s));
  // start block: random, low-pass filtered
  uint64_t rng_counter = 0;
  st = fill_random(c, w.V, b, opts.seed, rng_counter);
  if (st) return st;
  const double s_smooth = op.lam_min_sum - 1e-3 * hnorm;
  for (int it = 0; it < opts.smooth_start && opts.use_prec; ++it) {
    apply_prec_timed(c, w.V, w.P, b, s_smooth);
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.V, w.P, (size_t)b * N * sizeof(double),
                                      cudaMemcpyDeviceToDevice, s));
    stt.prec_applies += b;
  }
  const double thresh2 = (tol * hnorm) * (tol * hnorm);
  // the shift follows the lowest unconverged Ritz value on the device (TF32 preconditioner,
  // no fixed prec_shift); else it is fixed after the eager iterations
  const bool dev_shift = !std::isfinite(opts.prec_shift) && w.prec_dtype == TPS_TF32_TC;
  // eager iterations up to m = m_min; the shift follows the lowest Ritz value (fixed from
  // the last of them), the paper's -E0 when the caller fixes prec_shift
  double shift = opts.prec_shift;
  int m = 0;
  // with the shift on the device the iterations that fill m_min are captured too (their
  // sizes are static as well); else they run eagerly and fix the shift
  const int nfill = mmin / b;
  const int neager = dev_shift ? 0 : nfill;
  for (int e = 0; e < neager; ++e) {
    double sh = shift;
    if (!std::isfinite(sh)) {
      if (e == 0) {
        sh = s_smooth;
      } else {
        TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.h_pinned, w.theta, sizeof(double),
                                          cudaMemcpyDeviceToHost, s));
        TPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        const double th0 = w.h_pinned[0];
        sh = op.lam_min_sum - std::max(std::fabs(th0 - op.lam_min_sum), 1e-8 * hnorm);
      }
    }
    m = graph_iteration(c, GraphIter{m, false}, b, mmin, sh, opts.use_prec != 0, &stt.h_applies,
                        &stt.prec_applies, thresh2, hnorm, false);
    if (e == neager - 1) shift = sh;
  }
  if (opts.update_dtype == TPS_F64_TC) prewarm_update_split();
  // the captured cycle: m = 2b -> 3b, 3b -> 4b -> restart to 2b, inside a WHILE node
  const int max_outer = opts.max_outer > 0 ? opts.max_outer : 500;
  if (dev_shift) {
    shift = s_smooth;
    w.h_pinned[0] = shift;
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.gshift, w.h_pinned, sizeof(double), cudaMemcpyHostToDevice, s));
    TPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  }
  // graph construction takes driver locks; threads of a batch take turns
  static std::mutex build_mutex;
  std::unique_lock<std::mutex> build_lock(build_mutex);
  const auto t_build = std::chrono::steady_clock::now();
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto fail = [&](cudaError_t e, const char *what) {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    return cuda_error(ctx, e, what);
  };
  cudaError_t e = cudaGraphCreate(&graph, 0);
  if (e != cudaSuccess) return fail(e, "cudaGraphCreate");
  cudaGraphConditionalHandle loop;
  e = cudaGraphConditionalHandleCreate(&loop, graph, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return fail(e, "cudaGraphConditionalHandleCreate");
  // capture on a private stream (nothing runs during capture; the graph launches on s)
  if (!w.capture) {
    e = cudaStreamCreateWithFlags(&w.capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(e, "cudaStreamCreateWithFlags");
  }
  const cudaStream_t cs = w.capture;
  Ctx cc{ctx, op, w, cs, N};
  std::vector<cudaGraphNode_t> leaf;
  if (neager < nfill) {  // the filling iterations, captured into the top-level graph
    e = cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(e, "cudaStreamBeginCaptureToGraph (fill)");
    for (int e2 = neager; e2 < nfill; ++e2)
      m = graph_iteration(cc, GraphIter{m, false}, b, mmin, shift, opts.use_prec != 0,
                          &stt.h_applies, &stt.prec_applies, thresh2, hnorm, dev_shift);
    cudaGraph_t captured_fill = nullptr;
    const cudaError_t fe = cudaStreamEndCapture(cs, &captured_fill);
    e = fe != cudaSuccess ? fe : cudaGetLastError();
    if (e != cudaSuccess) return fail(e, "capturing the filling iterations");
    size_t nn = 0;
    e = cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess) e = cudaGraphGetNodes(graph, nodes.data(), &nn);
    for (size_t i = 0; i < nn && e == cudaSuccess; ++i) {
      size_t nd = 0;
      e = cudaGraphNodeGetDependentNodes(nodes[i], nullptr, nullptr, &nd);
      if (e == cudaSuccess && nd == 0) leaf.push_back(nodes[i]);
    }
    if (e != cudaSuccess) return fail(e, "reading the graph's last node");
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = loop;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  e = cudaGraphAddNode(&wnode, graph, leaf.empty() ? nullptr : leaf.data(), nullptr, leaf.size(),
                       &cp);
  if (e != cudaSuccess) return fail(e, "cudaGraphAddNode (while)");
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(e, "cudaStreamBeginCaptureToGraph");
  int hcount = 0, pcount = 0;
  int mc = graph_iteration(cc, GraphIter{mmin, false}, b, mmin, shift, opts.use_prec != 0, &hcount,
                           &pcount, thresh2, hnorm, dev_shift);
  launch_conv_check(w.nrm2, k_req, thresh2, w.gstate, max_outer, loop, 0, cs);
  mc = graph_iteration(cc, GraphIter{mc, true}, b, mmin, shift, opts.use_prec != 0, &hcount,
                       &pcount, thresh2, hnorm, dev_shift);
  launch_conv_check(w.nrm2, k_req, thresh2, w.gstate, max_outer, loop, 1, cs);
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cs, &captured);
  e = ce != cudaSuccess ? ce : cudaGetLastError();
  if (e != cudaSuccess) return fail(e, "capturing the outer iteration");
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) return fail(e, "cudaGraphInstantiate");
  build_lock.unlock();
  const auto t_run = std::chrono::steady_clock::now();
  stt.graph_build_ms = std::chrono::duration<double, std::milli>(t_run - t_build).count();
  e = cudaGraphLaunch(exec, s);
  if (e != cudaSuccess) return fail(e, "cudaGraphLaunch");
  int state[2] = {0, 0};
  e = cudaMemcpyAsync(w.hi_pinned, w.gstate, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(e, "running the outer-iteration graph");
  stt.graph_run_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() -
                                                               t_run).count();
  std::memcpy(state, w.hi_pinned, sizeof(state));
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  exec = nullptr;
  graph = nullptr;
  const int cycles = (state[1] + 1) / 2;
  stt.outer_iters = nfill + state[1];
  stt.h_applies += cycles * hcount;
  stt.prec_applies += cycles * pcount;
  stt.restarts = cycles;
  // results: Ritz values, vectors (QX) expanded to the full grid, signs fixed; the Ritz
  // vectors of a converged state are unit vectors (a dropped column would be zero)
  TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.h_pinned, w.theta, k * sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
  col_norms2(c, w.QX, k_req, w.ref);
  TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.h_pinned + 64, w.ref, k_req * sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
  TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.h_pinned + 128, w.nrm2, k_req * sizeof(double),
                                    cudaMemcpyDeviceToHost, s));
  TPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  bool ok = state[0] != 0;
  for (int i = 0; i < k_req && ok; ++i) ok = std::fabs(w.h_pinned[64 + i] - 1.0) <= 1e-8;
  if (!ok) return TPS_ERR_NOT_CONVERGED;  // the caller falls back to the host-driven loop
  for (int i = 0; i < k_req; ++i) {
    evals_host[i] = w.h_pinned[i];
    if (i < 64) stt.resid[i] = std::sqrt(std::max(w.h_pinned[128 + i], 0.0)) / hnorm;
    const double *src = w.QX + (long long)i * N;
    double *dst = evecs_dev + (long long)i * ctx->full.N;
    if (parity != TPS_ANY)
      launch_sector_expand(parity, ctx->n[0], ctx->n[1], 1, src, dst, s);
    else
      TPS_CUDA_TRY(ctx, cudaMemcpyAsync(dst, src, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  launch_fix_sign(k_req, ctx->full.N, evecs_dev, ctx->gscr, s);
  TPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  TPS_CUDA_TRY(ctx, cudaGetLastError());
  stt.n_converged = k_req;
  stt.kernel_launches = g_kernel_launches.load() - launches0;
  stt.time_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (stats) *stats = stt;
  {
    const int f = (w.h64_dtype == TPS_F64_TC ? tc_operator_status(op) : 0) |
                  (opts.update_dtype == TPS_F64_TC ? update_split_status() : 0);
    if (f < 0) return set_error(ctx, TPS_ERR_CUDA, "reading the device status flag failed");
    if (f) return set_error(ctx, TPS_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait");
  }
  return TPS_OK;
}

// ---------------------------------------------------------------------------------------
// Jacobi-Davidson for the non-symmetric H of the paper's own discretisation (Sec. 3.1: the
// mapped Chebyshev D2 is dense and non-symmetric; Sec. 4.1: JDQR).  The search space V is
// orthonormal; the projected matrix G = V^T H V is non-symmetric and kept whole (new
// columns V^T H T and new rows T^T H V per expansion); its k eigenpairs of smallest real
// part (host QR in complex arithmetic, m <= 64) give the Ritz pairs (theta_i, x_i = V y_i),
// whose residuals r_i = H x_i - theta_i x_i are orthogonal to V.  The correction equation
// Eq. jdcor is solved for the unconverged pairs with Qt an orthonormal basis of all k target
// Ritz vectors, with the Sec. 4.2 preconditioner (fast diagonalisation with S^-1 in place of
// S^T).  At restart V keeps an orthonormal basis of the lowest m_min Ritz vectors.  The k
// target pairs stay in the search space until all of them have converged (no locking).
int solve_nonsym_impl(tps_ctx *ctx, int k_req, int parity, double tol, int block,
                      const tps_solver_opts *opts_in, double *evals_host, double *evecs_dev,
                      tps_stats *stats, cudaStream_t s) {
  const auto t_start = std::chrono::steady_clock::now();
  tps_solver_opts opts;
  tps_default_opts(&opts);
  if (opts_in) opts = *opts_in;
  int k = k_req + std::max(0, opts.guard);
  const int b = std::min(block, k);
  int mmin = opts.m_min > 0 ? opts.m_min : std::max(2 * k, 8);
  mmin = ((mmin + b - 1) / b) * b;
  int mmax = opts.m_max > 0 ? opts.m_max : mmin + 2 * b;
  mmax = std::min(mmax, 64);
  if (mmin > mmax - b) mmin = std::max(b, mmax - b);
  if (mmin < k) mmin = std::min(k, mmax - b);
  const int steps = opts.inner_steps > 0 ? opts.inner_steps : 3;
  const int max_outer = opts.max_outer > 0 ? opts.max_outer : 500;
  const double inner_tol = opts.inner_tol > 0 ? opts.inner_tol : 1e-3;
  if (mmax < 2 * b || steps > 40 || k > mmin)
    return set_error(ctx, TPS_ERR_INVALID_ARG, "search space too small for k and the block");
  const DevOperator *opp = &ctx->full;
  if (parity != TPS_ANY) {
    int st = build_sector_operator(ctx, parity);
    if (st) return st;
    opp = &ctx->sect[parity];
  }
  const DevOperator &op = *opp;
  const long long N = op.N;
  if (k_req > N / 2) return set_error(ctx, TPS_ERR_INVALID_ARG, "k too large for the grid");
  int st = alloc_workspace(ctx, N, mmax, std::max(b, k), k, steps);
  if (st) return st;
  SolverWorkspace &w = *ctx->sw;
  Ctx c{ctx, op, w, s, N};
  w.tm.reset(opts.timing != 0);
  w.prec_dtype = opts.prec_dtype == TPS_F64 ? TPS_F64 : TPS_F32;
  w.corr_low = false;
  w.h64_dtype = opts.h64_dtype == TPS_F64_TC ? TPS_F64_TC : TPS_F64;
  if (w.h64_dtype == TPS_F64_TC) TPS_CUDA_TRY(ctx, ensure_tc_operator(op, s));
  struct Scope {
    explicit Scope(PhaseTiming *t) {
      tl_timing = t;
      tl_split_updates = false;  // the Ritz products stay FP64 (non-orthogonal Y)
      tl_split_grams = false;
    }
    ~Scope() { tl_timing = nullptr; }
  } scope(&w.tm);
  const long long launches0 = g_kernel_launches.load();
  double hnorm = 0.0;
  tps_get_info(ctx, nullptr, &hnorm);
  tps_stats stt;
  std::memset(&stt, 0, sizeof(stt));
  stt.hnorm_est = hnorm;
  const int ldG = w.mmax;
  std::vector<double> Gh((size_t)ldG * ldG), Gr((size_t)ldG * ldG), Yh((size_t)ldG * ldG);
  std::vector<double> lam(ldG, 0.0), res(k, 0.0);
  uint64_t rng_counter = 0;
  // random start block, low-pass filtered by the kinetic preconditioner
  st = fill_random(c, w.V, b, opts.seed, rng_counter);
  if (st) return st;
  const double s_smooth = op.lam_min_sum - 1e-3 * hnorm;
  for (int it = 0; it < opts.smooth_start && opts.use_prec; ++it) {
    apply_prec_timed(c, w.V, w.P, b, s_smooth);
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.V, w.P, (size_t)b * N * sizeof(double),
                                      cudaMemcpyDeviceToDevice, s));
    stt.prec_applies += b;
  }
  int m = 0, bn = b, outer = 0;
  bool converged = false;
  for (; outer < max_outer; ++outer) {
    // (1) orthonormalise the new block against V, (2) apply H, (3) extend G
    double *T = w.V + (long long)m * N;
    int rank = 0;
    for (int attempt = 0; attempt < 3; ++attempt) {
      st = orthonormalize(c, nullptr, 0, w.V, m, T, bn, &rank);
      if (st) return st;
      if (rank > 0) break;
      st = fill_random(c, T, bn, opts.seed, rng_counter);
      if (st) return st;
    }
    if (rank == 0) return set_error(ctx, TPS_ERR_NOT_CONVERGED, "search space cannot be expanded");
    double *HT = w.HV + (long long)m * N;
    apply_h_timed(c, T, HT, rank, nullptr, false);
    stt.h_applies += rank;
    tgram(w.V, N, 0, m + rank, HT, N, 0, rank, N, w.G + (long long)m * ldG, ldG, 0, 1, ctx->gscr, s);
    if (m > 0) tgram(T, N, 0, rank, w.HV, N, 0, m, N, w.G + m, ldG, 0, 1, ctx->gscr, s);
    m += rank;
    // (4) Ritz pairs of the non-symmetric G (host, complex QR)
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(Gh.data(), w.G, (size_t)ldG * m * sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
    TPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) Gr[(size_t)i * m + j] = Gh[(size_t)j * ldG + i];
    const int nk = std::min(m, std::max(k, mmin));
    double imag = 0.0;
    std::fill(Yh.begin(), Yh.end(), 0.0);
    if (complex_eig_lowest(m, Gr.data(), nk, lam.data(), Yh.data(), ldG, &imag))
      return set_error(ctx, TPS_ERR_NOT_CONVERGED, "Ritz eigenproblem did not converge");
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.Y, Yh.data(), (size_t)ldG * nk * sizeof(double),
                                      cudaMemcpyHostToDevice, s));
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.theta, lam.data(), nk * sizeof(double),
                                      cudaMemcpyHostToDevice, s));
    // (5) Ritz vectors, residuals and their norms for the k targets
    const int nt = std::min(k, m);
    tupdate(w.V, N, 0, m, w.Y, ldG, 0, nt, 1.0, 0.0, w.QX, N, 0, N, 1, s);
    tupdate(w.HV, N, 0, m, w.Y, ldG, 0, nt, 1.0, 0.0, w.HX, N, 0, N, 1, s);
    launch_residual(nt, N, w.HX, w.QX, w.theta, w.R, s);
    col_norms2(c, w.R, nt, w.nrm2);
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.h_pinned, w.nrm2, nt * sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
    TPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    TPS_CUDA_TRY(ctx, cudaGetLastError());
    w.tm.drain();
    int nconv = 0;
    std::vector<int> active;
    for (int i = 0; i < nt; ++i) {
      res[i] = std::sqrt(std::max(w.h_pinned[i], 0.0)) / hnorm;
      if (res[i] <= tol && std::fabs(imag) <= 1e-8 * std::max(1.0, std::fabs(lam[i])))
        ++nconv;
      else if ((int)active.size() < b)
        active.push_back(i);
    }
    if (nt == k && nconv == k) {
      converged = true;
      ++outer;
      break;
    }
    // (6) restart: an orthonormal basis of the lowest m_min Ritz vectors (host MGS of Y)
    if (m + b > mmax) {
      const int mk = std::min(mmin, nk);
      std::vector<double> Z((size_t)ldG * mk, 0.0);
      int r = 0;
      for (int j = 0; j < mk; ++j) {
        double *z = Z.data() + (size_t)r * ldG;
        for (int i = 0; i < m; ++i) z[i] = Yh[(size_t)j * ldG + i];
        for (int pass = 0; pass < 2; ++pass)
          for (int q = 0; q < r; ++q) {
            const double *zq = Z.data() + (size_t)q * ldG;
            double d = 0.0;
            for (int i = 0; i < m; ++i) d += zq[i] * z[i];
            for (int i = 0; i < m; ++i) z[i] -= d * zq[i];
          }
        double nz = 0.0;
        for (int i = 0; i < m; ++i) nz += z[i] * z[i];
        nz = std::sqrt(nz);
        if (nz < 1e-10) continue;
        for (int i = 0; i < m; ++i) z[i] /= nz;
        ++r;
      }
      // G in the new basis: Z^T G Z (host), V <- V Z, HV <- HV Z
      std::vector<double> GZ((size_t)m * r, 0.0), Gn((size_t)ldG * ldG, 0.0);
      for (int j = 0; j < r; ++j)
        for (int i = 0; i < m; ++i) {
          double a = 0.0;
          for (int l = 0; l < m; ++l) a += Gr[(size_t)i * m + l] * Z[(size_t)j * ldG + l];
          GZ[(size_t)j * m + i] = a;
        }
      for (int j = 0; j < r; ++j)
        for (int i = 0; i < r; ++i) {
          double a = 0.0;
          for (int l = 0; l < m; ++l) a += Z[(size_t)i * ldG + l] * GZ[(size_t)j * m + l];
          Gn[(size_t)j * ldG + i] = a;
        }
      TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.Arot, Z.data(), (size_t)ldG * r * sizeof(double),
                                        cudaMemcpyHostToDevice, s));
      tupdate(w.V, N, 0, m, w.Arot, ldG, 0, r, 1.0, 0.0, w.V2, N, 0, N, 1, s);
      tupdate(w.HV, N, 0, m, w.Arot, ldG, 0, r, 1.0, 0.0, w.HV2, N, 0, N, 1, s);
      std::swap(w.V, w.V2);
      std::swap(w.HV, w.HV2);
      TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.G, Gn.data(), (size_t)ldG * r * sizeof(double),
                                        cudaMemcpyHostToDevice, s));
      m = r;
      ++stt.restarts;
    }
    // (7) correction equations of the active pairs: Qt = orthonormal basis of the targets
    const int na = (int)active.size();
    if (na == 0) {  // every pair so far converged but fewer than k exist: widen with noise
      st = fill_random(c, w.V + (long long)m * N, b, opts.seed, rng_counter);
      if (st) return st;
      bn = b;
      continue;
    }
    for (int a = 0; a < na; ++a) {
      TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.P + (long long)a * N, w.R + (long long)active[a] * N,
                                        N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      w.h_pinned[256 + a] = lam[active[a]];
    }
    TPS_CUDA_TRY(ctx, cudaMemcpyAsync(w.theta2, w.h_pinned + 256, na * sizeof(double),
                                      cudaMemcpyHostToDevice, s));
    int nq = 0;
    st = orthonormalize(c, nullptr, 0, nullptr, 0, w.QX, nt, &nq);
    if (st) return st;
    double shift = opts.prec_shift;
    if (!std::isfinite(shift)) {
      const double th0 = lam[active[0]];
      shift = op.lam_min_sum - std::max(std::fabs(th0 - op.lam_min_sum), 1e-8 * hnorm);
    }
    st = correction_impl(ctx, op, w.QX, nq, nullptr, 0, w.P, w.theta2, na, steps, opts.use_prec,
                         shift, inner_tol, w.V + (long long)m * N, &stt.h_applies,
                         &stt.prec_applies, s, false, false);
    if (st) return st;
    stt.inner_steps += steps * na;
    bn = na;
  }
  stt.outer_iters = outer;
  // results: Ritz values ascending, vectors expanded to the full grid, signs fixed
  const int nret = converged ? k_req : 0;
  for (int i = 0; i < nret; ++i) {
    evals_host[i] = lam[i];
    if (i < 64) stt.resid[i] = res[i];
    const double *src = w.QX + (long long)i * N;
    double *dst = evecs_dev + (long long)i * ctx->full.N;
    if (parity != TPS_ANY)
      launch_mirror_expand(parity, ctx->n[0], ctx->n[1], 1, src, dst, s);
    else
      TPS_CUDA_TRY(ctx, cudaMemcpyAsync(dst, src, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (nret > 0) launch_fix_sign(nret, ctx->full.N, evecs_dev, ctx->gscr, s);
  TPS_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  TPS_CUDA_TRY(ctx, cudaGetLastError());
  w.tm.drain();
  stt.n_converged = nret;
  stt.h_ms = w.tm.ms[0];
  stt.prec_ms = w.tm.ms[1];
  stt.h_flops = w.tm.flops[0];
  stt.prec_flops = w.tm.flops[1];
  stt.h_launches = w.tm.launches[0];
  stt.prec_launches = w.tm.launches[1];
  stt.kernel_launches = g_kernel_launches.load() - launches0;
  stt.time_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (stats) *stats = stt;
  if (w.h64_dtype == TPS_F64_TC) {
    const int f = tc_operator_status(op);
    if (f < 0) return set_error(ctx, TPS_ERR_CUDA, "reading the device status flag failed");
    if (f) return set_error(ctx, TPS_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait");
  }
  if (!converged) return set_error(ctx, TPS_ERR_NOT_CONVERGED, "outer-iteration cap reached");
  return TPS_OK;
}

}  // namespace tps

using namespace tps;

extern "C" {

void tps_default_opts(tps_solver_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->use_prec = 1;
  o->prec_shift = NAN;
  o->seed = 12345;
  o->guard = 2;
  o->smooth_start = 2;
  o->prec_dtype = TPS_TF32_TC;  // TPS_F32 on 2D grids the TF32 passes do not take
  o->correction_dtype = TPS_F32;
  o->update_dtype = TPS_F64_TC;
  o->gram_dtype = TPS_F64_TC;
  o->h_dtype = TPS_F64;
  o->switch_tol = 1e-6;
  o->refine_block = 0;
  o->refine_inner_steps = 0;
  o->refine_inner_dtype = TPS_F64;
  o->h64_dtype = TPS_F64_TC;
}

int tps_solve(tps_ctx *ctx, int k, int parity, double tol, int block, const double *x0_dev,
              int n_x0, const tps_solver_opts *opts, double *evals_host, double *evecs_dev,
              tps_stats *stats, cudaStream_t stream) {
  if (!ctx) return TPS_ERR_INVALID_ARG;
  if (!ctx->have_masses || !ctx->have_grid)
    return set_error(ctx, TPS_ERR_NOT_CONFIGURED, "masses and grid must be set first");
  if (k < 1 || k > 64 || block < 1 || block > 32 || !(tol > 0) || !evals_host || !evecs_dev ||
      (parity != TPS_ANY && parity != TPS_X_EVEN && parity != TPS_X_ODD) || n_x0 < 0 ||
      (n_x0 > 0 && !x0_dev))
    return set_error(ctx, TPS_ERR_INVALID_ARG, "bad solve arguments");
  if (ctx->dim == 2 && parity != TPS_ANY)
    return set_error(ctx, TPS_ERR_INVALID_ARG, "2D supports TPS_ANY only");
  cudaSetDevice(ctx->device);
  if (ctx->grid_kind == 1) {
    if (n_x0 > 0) return set_error(ctx, TPS_ERR_INVALID_ARG, "no warm start on Chebyshev grids");
    return solve_nonsym_impl(ctx, k, parity, tol, block, opts, evals_host, evecs_dev, stats,
                             stream);
  }
  if (opts && opts->graph && n_x0 == 0 && ctx->dim == 1) {
    const int st = solve_graph_impl(ctx, k, parity, tol, *opts, evals_host, evecs_dev, stats,
                                    stream);
    if (st != TPS_ERR_NOT_CONVERGED) return st;
    // the graph's cycle did not converge within the cap (or returned a degenerate vector):
    // the host-driven loop solves the problem from scratch
  }
  return solve_impl(ctx, k, parity, tol, block, x0_dev, n_x0, opts, evals_host, evecs_dev, stats,
                    stream);
}

int tps_orthonormalize(tps_ctx *ctx, const double *Q_dev, long long ldq, int nq, double *T_dev,
                       long long ldt, int b, long long nrows, int *rank_host, cudaStream_t stream) {
  if (!ctx) return TPS_ERR_INVALID_ARG;
  if (b < 1 || b > 32 || nq < 0 || nq > 64 || nrows < 1 || ldq != nrows || ldt != nrows ||
      !T_dev || !rank_host || (nq > 0 && !Q_dev))
    return set_error(ctx, TPS_ERR_INVALID_ARG, "bad orthonormalize arguments (ld must equal nrows)");
  int st = alloc_workspace(ctx, nrows, std::max(nq, 2 * b), b, std::max(nq, 1), 1);
  if (st) return st;
  DevOperator dummy;
  dummy.N = nrows;
  Ctx c{ctx, dummy, *ctx->sw, stream, nrows};
  return orthonormalize(c, Q_dev, nq, nullptr, 0, T_dev, b, rank_host);
}

int tps_correction(tps_ctx *ctx, const double *Qt_dev, int nq, const double *R_dev,
                   const double *theta_dev, int nsys, int steps, int use_prec, double shift,
                   double *T_dev, cudaStream_t stream) {
  if (!ctx) return TPS_ERR_INVALID_ARG;
  if (!ctx->have_masses || !ctx->have_grid)
    return set_error(ctx, TPS_ERR_NOT_CONFIGURED, "masses and grid must be set first");
  if (nsys < 1 || nsys > 32 || nq < 0 || nq > 96 || steps < 1 || steps > 40 || !R_dev ||
      !theta_dev || !T_dev || (nq > 0 && !Qt_dev) || (use_prec && !std::isfinite(shift)))
    return set_error(ctx, TPS_ERR_INVALID_ARG, "bad correction arguments");
  int st = alloc_workspace(ctx, ctx->full.N, 2 * nsys, nsys, std::max(nq - nsys, 1), steps);
  if (st) return st;
  if (ctx->sw->kmax + ctx->sw->b < nq) {
    st = alloc_workspace(ctx, ctx->full.N, 2 * nsys, nsys, nq, steps);
    if (st) return st;
  }
  int ha = 0, pa = 0;
  ctx->sw->tm.reset(false);
  ctx->sw->prec_dtype = TPS_F64;
  ctx->sw->corr_low = false;
  st = correction_impl(ctx, ctx->full, Qt_dev, nq, nullptr, 0, R_dev, theta_dev, nsys, steps,
                       use_prec, shift, 0.0, T_dev, &ha, &pa, stream, false, false);
  if (st) return st;
  TPS_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
  return TPS_OK;
}

}  // extern "C"
