// api.cu -- the C entry points declared in include/randqr.h.
//
// Each factorization is a fixed sequence of kernels on the caller's stream; the host only
// checks arguments, carves the context's workspace and launches.  Launch sequence of
// rand_cholQR (Algorithm 3):
//   zero W1, Ws, G | (S2 once per (seed, s1, s2)) | CountSketch scatter V -> W1 |
//   sketch GEMM W1 -> Ws | Householder R_s of Ws | W = V R_s^{-1} (into Q) |
//   G = W^T W | R_c = chol(G), R = R_c R_s | Q = W R_c^{-1} (in place)
#include <stdio.h>
#include <string.h>

#include <new>

#include "common.cuh"

using rq::DevStatus;

namespace {

constexpr int64_t kMaxN = 128;

randqr_status cuda_fail(randqr_ctx *ctx, cudaError_t e, const char *where) {
  if (ctx) snprintf(ctx->last_err, sizeof(ctx->last_err), "%s: %s", where, cudaGetErrorString(e));
  return RANDQR_ERR_CUDA;
}

#define RQ_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

cudaEvent_t take_event(randqr_ctx *ctx) {
  if (!ctx->prof_pool.empty()) {
    cudaEvent_t e = ctx->prof_pool.back();
    ctx->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Launch through f(); when profiling is on, bracket it with events on s.
template <class F>
cudaError_t timed(randqr_ctx *ctx, cudaStream_t s, int kind, F &&f) {
  if (!ctx->prof) return f();
  cudaEvent_t b = take_event(ctx), e = take_event(ctx);
  if (!b || !e) return cudaErrorMemoryAllocation;
  cudaError_t r = cudaEventRecord(b, s);
  if (r != cudaSuccess) return r;
  r = f();
  if (r != cudaSuccess) return r;
  r = cudaEventRecord(e, s);
  ctx->prof_recs.push_back({kind, b, e});
  return r;
}

struct Workspace {
  double *W1, *Ws, *Rs, *G, *Rc, *Rt, *Rt2;
  float2 *Rdf, *rinv;  // pair form of the current triangular factor (RANDQR_F32X2)
  double *hq;          // multi-CTA Householder scratch (published reflectors, flags)
  double *acc;         // accuracy measurement: Q^T Q (packed), then the two residual sums
  double *blk;         // blocked solves (64 < n <= 128): five packed 64 x 64 blocks
};

size_t packed(int64_t n) { return (size_t)(n * (n + 1) / 2); }

size_t align_up(size_t b) { return (b + 255) & ~(size_t)255; }

// Ensure the slab holds `bytes`; grows by reallocation (after waiting for the device).
randqr_status ensure_ws(randqr_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return RANDQR_OK;
  if (ctx->budget && bytes + ctx->s2_bytes + ctx->hstage_bytes > ctx->budget) return RANDQR_ERR_NOMEM;
  RQ_CUDA(cudaDeviceSynchronize());
  if (ctx->ws) RQ_CUDA(cudaFree(ctx->ws));
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  if (cudaMalloc(&ctx->ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    return RANDQR_ERR_NOMEM;
  }
  ctx->ws_bytes = bytes;
  return RANDQR_OK;
}

// Ensure the staging area of randqr_factor_host holds `bytes` (same growth rule as the slab).
randqr_status ensure_host_stage(randqr_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->hstage_bytes) return RANDQR_OK;
  if (ctx->budget && bytes + ctx->ws_bytes + ctx->s2_bytes > ctx->budget) return RANDQR_ERR_NOMEM;
  RQ_CUDA(cudaDeviceSynchronize());
  if (ctx->hstage) RQ_CUDA(cudaFree(ctx->hstage));
  ctx->hstage = nullptr;
  ctx->hstage_bytes = 0;
  if (cudaMalloc(&ctx->hstage, bytes) != cudaSuccess) {
    cudaGetLastError();
    return RANDQR_ERR_NOMEM;
  }
  ctx->hstage_bytes = bytes;
  return RANDQR_OK;
}

size_t acc_doubles(int64_t n) { return packed(n) + 2; }
constexpr size_t kBlkDoubles = 5 * 2080;  // five packed 64 x 64 upper blocks

randqr_status carve(randqr_ctx *ctx, int64_t n, int64_t s1, int64_t s2, Workspace *w) {
  const size_t sz[12] = {align_up(sizeof(double) * (size_t)(s1 * n)),
                         align_up(sizeof(double) * (size_t)(s2 * n)),
                         align_up(sizeof(double) * packed(n)), align_up(sizeof(double) * packed(n)),
                         align_up(sizeof(double) * packed(n)), align_up(sizeof(double) * packed(n)),
                         align_up(sizeof(double) * packed(n)),
                         align_up(sizeof(float2) * rq::pack_df_elems(n)),
                         align_up(sizeof(float2) * rq::pack_df_rinv_elems(n)),
                         align_up(sizeof(double) * rq::hhqr_scratch_doubles(s2, n)),
                         align_up(sizeof(double) * acc_doubles(n)),
                         align_up(sizeof(double) * (n > 64 ? kBlkDoubles : 0))};
  size_t total = 0;
  for (size_t b : sz) total += b;
  randqr_status st = ensure_ws(ctx, total);
  if (st != RANDQR_OK) return st;
  char *p = (char *)ctx->ws;
  double **dst[7] = {&w->W1, &w->Ws, &w->Rs, &w->G, &w->Rc, &w->Rt, &w->Rt2};
  for (int i = 0; i < 7; ++i) {
    *dst[i] = (double *)p;
    p += sz[i];
  }
  w->Rdf = (float2 *)p;
  p += sz[7];
  w->rinv = (float2 *)p;
  p += sz[8];
  w->hq = (double *)p;
  p += sz[9];
  w->acc = (double *)p;
  p += sz[10];
  w->blk = (double *)p;
  return RANDQR_OK;
}

// The cached S2 for (seed, s1, s2), generated on `s` if missing.
randqr_status ensure_s2(randqr_ctx *ctx, uint64_t seed, int64_t s1, int64_t s2, cudaStream_t s,
                        const double **out) {
  if (!(ctx->s2_valid && ctx->s2_seed == seed && ctx->s2_s1 == s1 && ctx->s2_s2 == s2 &&
        ctx->s2_kind_cached == ctx->s2_kind)) {
    const size_t bytes = sizeof(double) * (size_t)(s1 * s2);
    if (bytes > ctx->s2_bytes) {
      if (ctx->budget && bytes + ctx->ws_bytes + ctx->hstage_bytes > ctx->budget) return RANDQR_ERR_NOMEM;
      RQ_CUDA(cudaDeviceSynchronize());
      if (ctx->s2_buf) RQ_CUDA(cudaFree(ctx->s2_buf));
      ctx->s2_buf = nullptr;
      ctx->s2_bytes = 0;
      if (cudaMalloc(&ctx->s2_buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return RANDQR_ERR_NOMEM;
      }
      ctx->s2_bytes = bytes;
    }
    RQ_CUDA(timed(ctx, s, rq::K_GAUSS_GEN, [&] {
      return ctx->s2_kind == RANDQR_SKETCH_RADEMACHER ? rq::launch_rad_gen(seed, s2, s1, ctx->s2_buf, s)
                                                      : rq::launch_gauss_gen(seed, s2, s1, ctx->s2_buf, s);
    }));
    ctx->s2_valid = true;
    ctx->s2_kind_cached = ctx->s2_kind;
    ctx->s2_seed = seed;
    ctx->s2_s1 = s1;
    ctx->s2_s2 = s2;
  }
  *out = ctx->s2_buf;
  return RANDQR_OK;
}

bool ranges_overlap(const void *a, size_t abytes, const void *b, size_t bbytes) {
  const char *pa = (const char *)a, *pb = (const char *)b;
  return pa < pb + bbytes && pb < pa + abytes;
}

size_t span_bytes(int64_t rows, int64_t cols, int64_t ld) {
  return rows == 0 ? 0 : sizeof(double) * (size_t)((rows - 1) * ld + cols);
}

// Common checks of the factorization entry points.
// A row shard (Sec. 4.1) may hold fewer rows than columns: `shard` relaxes m >= n to m >= 1.
bool bad_factor_args(const double *V, int64_t m, int64_t n, int64_t ldv, const double *Q,
                     int64_t ldq, const double *R, int64_t ldr, bool shard = false) {
  if (!V || !Q || !R) return true;
  if (n < 1 || n > kMaxN || m < (shard ? 1 : n) || ldv < n || ldq < n || ldr < n) return true;
  if ((const void *)Q != (const void *)V &&
      ranges_overlap(V, span_bytes(m, n, ldv), Q, span_bytes(m, n, ldq)))
    return true;
  if (Q == V && ldq != ldv) return true;
  if (ranges_overlap(R, span_bytes(n, n, ldr), Q, span_bytes(m, n, ldq)) ||
      ranges_overlap(R, span_bytes(n, n, ldr), V, span_bytes(m, n, ldv)))
    return true;
  return false;
}

bool bad_sketch_sizes(int64_t n, int64_t s1, int64_t s2) {
  return s2 < n || s1 < s2 || s1 >= ((int64_t)1 << 31) || s2 > ((int64_t)1 << 20);
}

// The single-sketch kinds fix one size: S2 = I needs s2 == s1, S1 = I needs s1 == m (and no
// row offset: a row block of V does not carry its columns of a dense S2).
bool bad_sketch_kind(const randqr_ctx *ctx, int64_t m, int64_t s1, int64_t s2, int64_t row0) {
  if (ctx->s2_kind == RANDQR_SKETCH_COUNT_ONLY) return s2 != s1;
  if (ctx->s2_kind == RANDQR_SKETCH_GAUSSIAN_ONLY) return s1 != m || row0 != 0;
  return false;
}

randqr_status begin_call(randqr_ctx *ctx, cudaStream_t s) {
  RQ_CUDA(cudaSetDevice(ctx->device));
  RQ_CUDA(rq::launch_status_reset(ctx->status_dev, ctx->wait_limit < 0 ? 0 : ctx->wait_limit + 1, s));
  return RANDQR_OK;
}

randqr_status finish_call(randqr_ctx *ctx, cudaStream_t s, randqr_info *info) {
  if (!info) return RANDQR_OK;
  return randqr_get_status(ctx, s, info);
}

}  // namespace

namespace rq {
bool factor_args_bad(const double *V, int64_t m, int64_t n, int64_t ldv, const double *Q, int64_t ldq,
                     const double *R, int64_t ldr) {
  return bad_factor_args(V, m, n, ldv, Q, ldq, R, ldr);
}
}  // namespace rq

// ---- Accuracy of a result (randqr_info.want_accuracy) -------------------------------------
// Enqueued after a factorization on its stream: Q^T Q into w.acc (packed) with the library's
// Gram (split products on the tensor cores where the method uses them, FP64 otherwise), and,
// when V is still intact, the residual sums ||V - Q R||_F^2, ||V||_F^2 after it; then the block
// is copied to the context's pinned host buffer.  Kernels skip themselves if the factorization
// failed (status word).  rq_accuracy_finish() turns the copy into the two numbers.
bool rq_accuracy_has_resid(const double *V, const double *Q);

randqr_status rq_accuracy_enqueue(randqr_ctx *ctx, const double *V, int64_t ldv, const double *Q, int64_t ldq,
                                  const double *R, int64_t ldr, int64_t m, int64_t n, cudaStream_t s) {
  if (!ctx->acc_host) {
    if (cudaMallocHost(&ctx->acc_host, sizeof(double) * acc_doubles(kMaxN)) != cudaSuccess) {
      cudaGetLastError();
      ctx->acc_host = nullptr;
      return RANDQR_ERR_NOMEM;
    }
  }
  Workspace w;
  randqr_status st = carve(ctx, n, 1, 1, &w);
  if (st != RANDQR_OK) return st;
  double *G = w.acc, *sums = w.acc + packed(n);
  RQ_CUDA(cudaMemsetAsync(w.acc, 0, sizeof(double) * acc_doubles(n), s));
  if (ctx->use_tc && rq::gram_oz_supported(n)) {
    RQ_CUDA(timed(ctx, s, rq::K_GRAM_TC, [&] {
      if (rq::gram_split_supported(n))
        return rq::launch_gram_split(Q, false, ldq, m, n, G, ctx->num_sms, ctx->status_dev, s);
      return rq::launch_gram_oz(Q, false, ldq, m, n, G, true, ctx->num_sms, ctx->status_dev, s);
    }));
  } else {
    RQ_CUDA(timed(ctx, s, rq::K_GRAM, [&] {
      return rq::launch_gram(Q, ldq, m, n, G, RANDQR_FP64, ctx->num_sms, ctx->status_dev, s);
    }));
  }
  if (rq_accuracy_has_resid(V, Q)) {
    RQ_CUDA(timed(ctx, s, rq::K_UNPACK, [&] { return rq::launch_pack_upper(R, ldr, n, w.Rt, ctx->status_dev, s); }));
    if (ctx->use_tc && rq::trsm_oz_supported(n)) {
      RQ_CUDA(timed(ctx, s, rq::K_TRSM_TC, [&] {
        return rq::launch_trsm_oz_resid(Q, ldq, V, ldv, m, n, w.Rt, sums, ctx->num_sms, ctx->status_dev, s);
      }));
    } else {
      RQ_CUDA(timed(ctx, s, rq::K_TRSM, [&] {
        return rq::launch_resid_f64(V, ldv, Q, ldq, m, n, w.Rt, sums, ctx->num_sms, ctx->status_dev, s);
      }));
    }
  }
  RQ_CUDA(cudaMemcpyAsync(ctx->acc_host, w.acc, sizeof(double) * acc_doubles(n), cudaMemcpyDeviceToHost, s));
  return RANDQR_OK;
}

bool rq_accuracy_has_resid(const double *V, const double *Q) { return V && (const void *)V != (const void *)Q; }

// After the stream has passed the copy: fill the accuracy fields of *info (the residual only
// when V was intact, rq_accuracy_has_resid).
void rq_accuracy_finish(randqr_ctx *ctx, int64_t n, bool have_resid, randqr_info *info) {
  const double *h = ctx->acc_host;
  info->orth_err2 = rq::sym_identity_gap2(h, (int)n);
  const double r2 = h[packed(n)], v2 = h[packed(n) + 1];
  info->resid_relF = (!have_resid || !(v2 > 0.0)) ? -1.0 : sqrt(r2 / v2);
}

namespace {

void clear_accuracy(randqr_info *info) {
  if (!info) return;
  info->orth_err2 = -1.0;
  info->resid_relF = -1.0;
}

// finish_call for the factorizations: with info->want_accuracy, measure the result first.
randqr_status finish_factor(randqr_ctx *ctx, cudaStream_t s, randqr_info *info, const double *V, int64_t ldv,
                            const double *Q, int64_t ldq, const double *R, int64_t ldr, int64_t m, int64_t n) {
  if (!info) return RANDQR_OK;
  clear_accuracy(info);
  const bool want = info->want_accuracy != 0;
  if (want) {
    randqr_status st = rq_accuracy_enqueue(ctx, V, ldv, Q, ldq, R, ldr, m, n, s);
    if (st != RANDQR_OK) return st;
  }
  randqr_status st = randqr_get_status(ctx, s, info);
  if (st == RANDQR_OK && want) rq_accuracy_finish(ctx, n, rq_accuracy_has_resid(V, Q), info);
  return st;
}

// Algorithm 1 steps 1-2 into w.Rs (packed); V read once by the scatter.
randqr_status sketch_and_hhqr(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                              int64_t ldv, int64_t s1, int64_t s2, uint64_t seed,
                              const double *S2, const Workspace &w, cudaStream_t s,
                              bool do_hhqr, int64_t row0 = 0) {
  if (ctx->s2_kind == RANDQR_SKETCH_COUNT_ONLY) {
    // single CountSketch (S2 = I, s2 == s1): the scatter goes straight into Ws
    RQ_CUDA(cudaMemsetAsync(w.Ws, 0, sizeof(double) * (size_t)(s2 * n), s));
    RQ_CUDA(timed(ctx, s, rq::K_CS_SCATTER, [&] {
      return rq::launch_cs_scatter(V, m, n, ldv, s1, seed, row0, w.Ws, ctx->num_sms, ctx->status_dev, s);
    }));
    if (do_hhqr)
      RQ_CUDA(timed(ctx, s, rq::K_HHQR, [&] { return rq::launch_hhqr(w.Ws, s2, n, w.Rs, w.hq, ctx->status_dev, s); }));
    return RANDQR_OK;
  }
  const double *S2p = S2;
  // a Rademacher S2 on the tensor-core path is generated inside the sketch GEMM: no buffer
  const bool rad_fly = !S2p && ctx->s2_kind == RANDQR_SKETCH_RADEMACHER && ctx->use_tc && rq::sketch_oz_supported(n);
  if (!S2p && !rad_fly) {
    randqr_status st = ensure_s2(ctx, seed + 1, s1, s2, s, &S2p);
    if (st != RANDQR_OK) return st;
  }
  if (ctx->s2_kind == RANDQR_SKETCH_GAUSSIAN_ONLY) {
    // single Gaussian sketch (S1 = I, s1 == m): Ws = S2 V, V packed to ld n in W1 if needed
    const double *B = V;
    if (ldv != n) {
      RQ_CUDA(cudaMemcpy2DAsync(w.W1, sizeof(double) * (size_t)n, V, sizeof(double) * (size_t)ldv,
                                sizeof(double) * (size_t)n, (size_t)m, cudaMemcpyDeviceToDevice, s));
      B = w.W1;
    }
    RQ_CUDA(cudaMemsetAsync(w.Ws, 0, sizeof(double) * (size_t)(s2 * n), s));
    RQ_CUDA(timed(ctx, s, rq::K_SKETCH_GEMM, [&] {
      return rq::launch_sketch_gemm(S2p, B, s2, s1, n, w.Ws, ctx->use_tc, ctx->num_sms, ctx->status_dev, s);
    }));
    if (do_hhqr)
      RQ_CUDA(timed(ctx, s, rq::K_HHQR, [&] { return rq::launch_hhqr(w.Ws, s2, n, w.Rs, w.hq, ctx->status_dev, s); }));
    return RANDQR_OK;
  }
  RQ_CUDA(cudaMemsetAsync(w.W1, 0, sizeof(double) * (size_t)(s1 * n), s));
  RQ_CUDA(cudaMemsetAsync(w.Ws, 0, sizeof(double) * (size_t)(s2 * n), s));
  RQ_CUDA(timed(ctx, s, rq::K_CS_SCATTER, [&] {
    return rq::launch_cs_scatter(V, m, n, ldv, s1, seed, row0, w.W1, ctx->num_sms, ctx->status_dev, s);
  }));
  RQ_CUDA(timed(ctx, s, rq::K_SKETCH_GEMM, [&] {
    if (rad_fly) return rq::launch_sketch_oz_rademacher(seed + 1, w.W1, n, s2, s1, n, w.Ws, ctx->num_sms, ctx->status_dev, s);
    return rq::launch_sketch_gemm(S2p, w.W1, s2, s1, n, w.Ws, ctx->use_tc, ctx->num_sms, ctx->status_dev, s);
  }));
  if (do_hhqr)
    RQ_CUDA(timed(ctx, s, rq::K_HHQR, [&] { return rq::launch_hhqr(w.Ws, s2, n, w.Rs, w.hq, ctx->status_dev, s); }));
  return RANDQR_OK;
}

// The split-product solves blocked for 64 < n <= 128 (n even, 16-byte aligned rows): columns split
// at n1 = n - 64 into X = [X1 X2], B = [[B11, B12], [0, B22]] upper triangular; every block
// product is one launch of the split-product kernel on at most 64 x 64 operands.  The dense block
// B12 (n1 x 64) runs as one product that leaves out its rows 32 .. n1 - 1 in columns 0 .. 31
// (the kernel's first column half takes K < 32), plus one half-width product that adds
// X1[:, 32:n1] B12[32:n1, 0:32] (only when n1 > 32).
bool blocked_tc_ok(const randqr_ctx *ctx, int64_t n, const void *X, int64_t ldx, const void *Y, int64_t ldy) {
  return ctx->use_tc && n > 64 && n <= 128 && n % 2 == 0 && ((uintptr_t)X & 15) == 0 && ((uintptr_t)Y & 15) == 0 &&
         ldx % 2 == 0 && ldy % 2 == 0;
}

// Y2 += X1 B12 for a dense n1 x 64 block B12 (row-major, ld 64): the full product without
// B12[32:n1, 0:32], then that corner as a half-width product into Y2's first 32 columns.
cudaError_t dense_block_add(randqr_ctx *ctx, const double *X1, int64_t ldx, double *Y2, int64_t ldy, int64_t m,
                            int64_t n1, const double *B12, cudaStream_t s) {
  cudaError_t e = timed(ctx, s, rq::K_TRSM_TC, [&] {
    return rq::launch_trsm_oz_block(X1, ldx, Y2, ldy, m, n1, 64, B12, false, Y2, ldy, ctx->num_sms, ctx->status_dev,
                                    s, 64);
  });
  if (e != cudaSuccess || n1 <= 32) return e;
  return timed(ctx, s, rq::K_TRSM_TC, [&] {
    return rq::launch_trsm_oz_block(X1 + 32, ldx, Y2, ldy, m, n1 - 32, 32, B12 + 32 * 64, false, Y2, ldy, ctx->num_sms,
                                    ctx->status_dev, s, 64);
  });
}

// Y = X Binv with Binv = R^{-1}, R well conditioned, by the explicit inverse (packed in Binv): all
// blocks are O(1) products, so the block sums may round separately.  Order: Y2 first (reads X2,
// X1), then Y1 (reads X1), so Y == X works in place.
randqr_status blocked_product_tc(randqr_ctx *ctx, const double *X, int64_t ldx, double *Y, int64_t ldy, int64_t m,
                                 int64_t n, const double *Binv, const Workspace &w, cudaStream_t s) {
  const int64_t n1 = n - 64;
  double *B22 = w.blk, *B12 = w.blk + 2080;  // B12 dense, n1 x 64 (ld 64)
  RQ_CUDA(rq::launch_block_prep(Binv, n, 0, 1.0, B22, ctx->status_dev, s));
  RQ_CUDA(rq::launch_block_prep(Binv, n, 3, 1.0, B12, ctx->status_dev, s));
  RQ_CUDA(timed(ctx, s, rq::K_TRSM_TC, [&] {
    return rq::launch_trsm_oz_block(X + n1, ldx, Y + n1, ldy, m, 64, 64, B22, false, nullptr, 0, ctx->num_sms,
                                    ctx->status_dev, s);
  }));
  RQ_CUDA(dense_block_add(ctx, X, ldx, Y + n1, ldy, m, n1, B12, s));
  RQ_CUDA(timed(ctx, s, rq::K_TRSM_TC, [&] {
    return rq::launch_trsm_oz_block(X, ldx, Y, ldy, m, n1, n1, Binv, false, nullptr, 0, ctx->num_sms,
                                    ctx->status_dev, s);
  }));
  return RANDQR_OK;
}

// W = V R_s^{-1} blocked, for an R_s that may be as ill conditioned as V: the inverse is applied
// only to the diagonal blocks, the off-diagonal block by substitution order,
//   W1 = V1 R11^{-1},   T = V2 - W1 R12,   W2 = T R22^{-1},
// each block product exact up to the split format and T formed as one rounded sum per term, a
// backward error of the size of a triangular solve's (row-wise, relative to |V| + |W1| |R12|).
randqr_status blocked_first_solve_tc(randqr_ctx *ctx, const double *V, int64_t ldv, double *Q, int64_t ldq, int64_t m,
                                     int64_t n, const double *Rs, const Workspace &w, cudaStream_t s) {
  const int64_t n1 = n - 64;
  double *R22 = w.blk, *mR12 = w.blk + 2080, *R11i = w.blk + 3 * 2080, *R22i = w.blk + 4 * 2080;
  RQ_CUDA(timed(ctx, s, rq::K_TRI_INV, [&] { return rq::launch_tri_inv(Rs, n1, R11i, ctx->status_dev, s); }));
  RQ_CUDA(rq::launch_block_prep(Rs, n, 0, 1.0, R22, ctx->status_dev, s));
  RQ_CUDA(timed(ctx, s, rq::K_TRI_INV, [&] { return rq::launch_tri_inv(R22, 64, R22i, ctx->status_dev, s); }));
  RQ_CUDA(rq::launch_block_prep(Rs, n, 3, -1.0, mR12, ctx->status_dev, s));  // -R12, dense
  RQ_CUDA(timed(ctx, s, rq::K_TRSM_TC, [&] {
    return rq::launch_trsm_oz_block(V, ldv, Q, ldq, m, n1, n1, R11i, false, nullptr, 0, ctx->num_sms, ctx->status_dev, s);
  }));
  // T = V2 - W1 R12 into Q2
  RQ_CUDA(timed(ctx, s, rq::K_TRSM_TC, [&] {
    return rq::launch_trsm_oz_block(Q, ldq, Q + n1, ldq, m, n1, 64, mR12, false, V + n1, ldv, ctx->num_sms,
                                    ctx->status_dev, s, 64);
  }));
  if (n1 > 32) {
    RQ_CUDA(timed(ctx, s, rq::K_TRSM_TC, [&] {
      return rq::launch_trsm_oz_block(Q + 32, ldq, Q + n1, ldq, m, n1 - 32, 32, mR12 + 32 * 64, false, Q + n1, ldq,
                                      ctx->num_sms, ctx->status_dev, s, 64);
    }));
  }
  RQ_CUDA(timed(ctx, s, rq::K_TRSM_TC, [&] {
    return rq::launch_trsm_oz_block(Q + n1, ldq, Q + n1, ldq, m, 64, 64, R22i, false, nullptr, 0, ctx->num_sms,
                                    ctx->status_dev, s);
  }));
  return RANDQR_OK;
}

// Y = X R_c^{-1} as the product X (R_c^{-1}) on the tensor cores, R_c^{-1} computed by column
// back substitution into w.Rt2 (after the Cholesky kernel has read R_c).  The computed inverse
// perturbs Y on the right by I + F with ||F|| of order n u kappa(R_c): used for the Cholesky
// passes (R_c well conditioned in rand_cholQR; kappa(R_c) <= about u^{-1/2} in the baselines).
randqr_status solve_by_inverse_tc(randqr_ctx *ctx, const double *X, int64_t ldx, double *Y,
                                  int64_t ldy, int64_t m, int64_t n, const Workspace &w,
                                  cudaStream_t s, int digits = 7) {
  if (n > 64) {
    RQ_CUDA(timed(ctx, s, rq::K_TRI_INV, [&] { return rq::launch_tri_inv(w.Rc, n, w.Rt2, ctx->status_dev, s); }));
    return blocked_product_tc(ctx, X, ldx, Y, ldy, m, n, w.Rt2, w, s);
  }
  RQ_CUDA(timed(ctx, s, rq::K_TRI_INV, [&] { return rq::launch_tri_inv(w.Rc, n, w.Rt2, ctx->status_dev, s); }));
  RQ_CUDA(timed(ctx, s, rq::K_TRSM_TC, [&] {
    return rq::launch_trsm_oz(X, ldx, Y, ldy, m, n, w.Rt2, ctx->num_sms, ctx->status_dev, s, digits);
  }));
  return RANDQR_OK;
}

bool use_tc_solve(const randqr_ctx *ctx, int64_t n) { return ctx->use_tc && rq::trsm_oz_supported(n); }

// G += X^T X on the tensor cores: the pipelined kernel for n <= 64, the older one up to 128.
cudaError_t launch_gram_tc(const randqr_ctx *ctx, const void *X, bool x_df, int64_t ldx, int64_t m,
                           int64_t n, double *G, cudaStream_t s) {
  if (rq::gram_split_supported(n))
    return rq::launch_gram_split(X, x_df, ldx, m, n, G, ctx->num_sms, ctx->status_dev, s);
  if (!x_df && n > 64 && n <= 128) {
    // the first 64 columns' Gram, then the columns 64 .. n - 1 against all n (upper triangle)
    cudaError_t e = rq::launch_gram_split(X, false, ldx, m, 64, G, ctx->num_sms, ctx->status_dev, s);
    if (e != cudaSuccess) return e;
    return rq::launch_gram_cross((const double *)X, ldx, m, n, G, ctx->num_sms, ctx->status_dev, s);
  }
  return rq::launch_gram_oz(X, x_df, ldx, m, n, G, !x_df, ctx->num_sms, ctx->status_dev, s);
}

// One cholQR pass (Algorithm 2) on X into Y: G = X^T X (+ shift) -> R_x -> Y = X R_x^{-1}.
// With Rprev, writes Rnext = R_x Rprev (packed); with Rdense, writes that product (or R_x)
// dense.  inverse_ok: the solve may be the tensor-core product with R_x^{-1}.
randqr_status cholqr_pass(randqr_ctx *ctx, const double *X, int64_t ldx, double *Y, int64_t ldy,
                          int64_t m, int64_t n, double shift_coeff, const double *Rprev,
                          double *Rnext, double *Rdense, int64_t ldr, int stage,
                          randqr_precision prec, const Workspace &w, cudaStream_t s,
                          bool inverse_ok = false, int digits = 7, bool gram_done = false) {
  if (!gram_done) {  // (gram_done: G = X^T X is already in w.G, formed by the fused first pass)
    RQ_CUDA(cudaMemsetAsync(w.G, 0, sizeof(double) * packed(n), s));
    if (ctx->use_tc && rq::gram_oz_supported(n)) {
      RQ_CUDA(timed(ctx, s, rq::K_GRAM_TC, [&] {
        return launch_gram_tc(ctx, X, false, ldx, m, n, w.G, s);
      }));
    } else {
      RQ_CUDA(timed(ctx, s, rq::K_GRAM, [&] {
        return rq::launch_gram(X, ldx, m, n, w.G, prec, ctx->num_sms, ctx->status_dev, s);
      }));
    }
  }
  RQ_CUDA(timed(ctx, s, rq::K_POTRF, [&] {
    return rq::launch_potrf(w.G, n, shift_coeff, w.Rc, Rprev, Rnext, Rdense, ldr, stage,
                            ctx->status_dev, s);
  }));
  if (inverse_ok && (use_tc_solve(ctx, n) || blocked_tc_ok(ctx, n, X, ldx, Y, ldy)))
    return solve_by_inverse_tc(ctx, X, ldx, Y, ldy, m, n, w, s, digits);
  RQ_CUDA(timed(ctx, s, rq::K_TRSM, [&] {
    return rq::launch_trsm(X, ldx, Y, ldy, m, n, w.Rc, prec, ctx->num_sms, ctx->status_dev, s);
  }));
  return RANDQR_OK;
}

}  // namespace

extern "C" {

randqr_status randqr_create(randqr_ctx **ctx_out, int device, size_t hbm_budget_bytes) {
  if (!ctx_out) return RANDQR_ERR_ARG;
  *ctx_out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return RANDQR_ERR_ARG;
  }
  randqr_ctx *ctx = new (std::nothrow) randqr_ctx();
  if (!ctx) return RANDQR_ERR_NOMEM;
  ctx->device = device;
  ctx->budget = hbm_budget_bytes;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&ctx->status_dev, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost(&ctx->status_host, sizeof(DevStatus)) != cudaSuccess ||
      cudaMemset(ctx->status_dev, 0, sizeof(DevStatus)) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->status_dev) cudaFree(ctx->status_dev);
    if (ctx->status_host) cudaFreeHost(ctx->status_host);
    delete ctx;
    return RANDQR_ERR_CUDA;
  }
  *ctx_out = ctx;
  return RANDQR_OK;
}

randqr_status randqr_destroy(randqr_ctx *ctx) {
  if (!ctx) return RANDQR_ERR_ARG;
  cudaSetDevice(ctx->device);
  rq_server_destroy(ctx);
  rq_batcher_destroy(ctx);
  cudaDeviceSynchronize();
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->hstage) cudaFree(ctx->hstage);
  if (ctx->s2_buf) cudaFree(ctx->s2_buf);
  if (ctx->status_dev) cudaFree(ctx->status_dev);
  if (ctx->status_host) cudaFreeHost(ctx->status_host);
  if (ctx->acc_host) cudaFreeHost(ctx->acc_host);
  for (auto &r : ctx->prof_recs) {
    cudaEventDestroy(r.beg);
    cudaEventDestroy(r.end);
  }
  for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
  delete ctx;
  return RANDQR_OK;
}

randqr_status randqr_set_tensor_cores(randqr_ctx *ctx, int enable) {
  if (!ctx) return RANDQR_ERR_ARG;
  if (ctx->use_tc != (enable != 0) && ctx->batcher) rq_batcher_destroy(ctx);  // graphs hold the old kernels
  ctx->use_tc = enable != 0;
  return RANDQR_OK;
}

randqr_status randqr_set_fused_first_pass(randqr_ctx *ctx, int enable) {
  if (!ctx) return RANDQR_ERR_ARG;
  if (ctx->fuse_first_pass != (enable != 0) && ctx->batcher) rq_batcher_destroy(ctx);  // graphs hold the old kernels
  ctx->fuse_first_pass = enable != 0;
  return RANDQR_OK;
}

randqr_status randqr_set_wait_limit(randqr_ctx *ctx, int32_t polls) {
  if (!ctx) {
    rq_static_set_wait_limit(polls);
    return RANDQR_OK;
  }
  const int32_t limit = polls < 0 ? -1 : std::min<int32_t>(polls, (1 << 30) - 1);
  if (limit != ctx->wait_limit && ctx->batcher) rq_batcher_destroy(ctx);  // graphs hold the old bound
  ctx->wait_limit = limit;
  return RANDQR_OK;
}

randqr_status randqr_set_profiling(randqr_ctx *ctx, int enable) {
  if (!ctx) return RANDQR_ERR_ARG;
  ctx->prof = enable != 0;
  return RANDQR_OK;
}

randqr_status randqr_get_kernel_times(randqr_ctx *ctx, int32_t max_kinds, double *total_ms,
                                      int64_t *launches, int32_t *n_kinds) {
  if (!ctx || max_kinds < 0 || (max_kinds > 0 && (!total_ms || !launches))) return RANDQR_ERR_ARG;
  RQ_CUDA(cudaSetDevice(ctx->device));
  const int nk = std::min<int>(max_kinds, rq::K_NUM_KINDS);
  for (int k = 0; k < nk; ++k) {
    total_ms[k] = 0.0;
    launches[k] = 0;
  }
  randqr_status st = RANDQR_OK;
  for (auto &r : ctx->prof_recs) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(r.end);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.beg, r.end);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "cudaEventElapsedTime");
    if (r.kind < nk) {
      total_ms[r.kind] += ms;
      launches[r.kind] += 1;
    }
    ctx->prof_pool.push_back(r.beg);
    ctx->prof_pool.push_back(r.end);
  }
  ctx->prof_recs.clear();
  if (n_kinds) *n_kinds = nk;
  return st;
}

const char *randqr_kernel_name(int32_t kind) {
  static const char *names[rq::K_NUM_KINDS] = {"gauss_gen", "cs_scatter", "sketch_gemm", "hhqr",
                                               "trsm", "gram", "potrf", "unpack", "cs_hash",
                                               "pack_df", "trsm_df", "gram_df", "gram_tc",
                                               "tri_inv", "trsm_tc", "solve_gram"};
  return (kind >= 0 && kind < rq::K_NUM_KINDS) ? names[kind] : "unknown";
}

const char *randqr_status_string(randqr_status s) {
  switch (s) {
    case RANDQR_OK: return "ok";
    case RANDQR_PENDING: return "pending";
    case RANDQR_ERR_ARG: return "invalid argument";
    case RANDQR_ERR_NOT_SPD: return "Cholesky breakdown (Gram matrix not numerically positive definite)";
    case RANDQR_ERR_RANK: return "zero or non-finite diagonal in the sketch's triangular factor";
    case RANDQR_ERR_NONFINITE: return "non-finite value";
    case RANDQR_ERR_NOMEM: return "out of device memory or over the HBM budget";
    case RANDQR_ERR_ADMISSION: return "request can never fit the HBM budget";
    case RANDQR_ERR_TIMEOUT: return "bounded device wait timed out";
    case RANDQR_ERR_CUDA: return "CUDA runtime error";
    case RANDQR_ERR_TICKET: return "unknown ticket";
  }
  return "unknown status";
}

const char *randqr_last_cuda_error(const randqr_ctx *ctx) { return ctx ? ctx->last_err : ""; }

size_t randqr_workspace_bytes(const randqr_ctx *ctx) {
  return ctx ? ctx->ws_bytes + ctx->s2_bytes : 0;
}

randqr_status randqr_get_status(randqr_ctx *ctx, void *stream, randqr_info *info) {
  if (!ctx) return RANDQR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  RQ_CUDA(cudaSetDevice(ctx->device));
  RQ_CUDA(cudaMemcpyAsync(ctx->status_host, ctx->status_dev, sizeof(DevStatus),
                          cudaMemcpyDeviceToHost, s));
  RQ_CUDA(cudaStreamSynchronize(s));
  const DevStatus h = *ctx->status_host;
  if (info) {
    info->info = h.info;
    info->stage = h.stage;
    info->rs_min_diag = h.dmin;
    info->rs_max_diag = h.dmax;
  }
  return (randqr_status)h.code;
}

randqr_status randqr_cs_hash(randqr_ctx *ctx, uint64_t seed, int64_t m, int64_t s1,
                             int32_t *bucket_dev, int8_t *sign_dev, void *stream) {
  if (!ctx || m < 0 || s1 < 1 || s1 >= ((int64_t)1 << 31) || (m > 0 && (!bucket_dev || !sign_dev)))
    return RANDQR_ERR_ARG;
  RQ_CUDA(cudaSetDevice(ctx->device));
  RQ_CUDA(timed(ctx, (cudaStream_t)stream, rq::K_CS_HASH, [&] {
    return rq::launch_cs_hash(seed, m, s1, bucket_dev, sign_dev, (cudaStream_t)stream);
  }));
  return RANDQR_OK;
}

randqr_status randqr_gauss_sketch(randqr_ctx *ctx, uint64_t seed, int64_t s2, int64_t s1,
                                  double *S2_dev, void *stream) {
  if (!ctx || !S2_dev || s2 < 1 || s1 < 1) return RANDQR_ERR_ARG;
  RQ_CUDA(cudaSetDevice(ctx->device));
  RQ_CUDA(timed(ctx, (cudaStream_t)stream, rq::K_GAUSS_GEN, [&] {
    return rq::launch_gauss_gen(seed, s2, s1, S2_dev, (cudaStream_t)stream);
  }));
  return RANDQR_OK;
}

randqr_status randqr_rademacher_sketch(randqr_ctx *ctx, uint64_t seed, int64_t s2, int64_t s1,
                                      double *S2_dev, void *stream) {
  if (!ctx || !S2_dev || s2 < 1 || s1 < 1) return RANDQR_ERR_ARG;
  RQ_CUDA(cudaSetDevice(ctx->device));
  RQ_CUDA(timed(ctx, (cudaStream_t)stream, rq::K_GAUSS_GEN, [&] {
    return rq::launch_rad_gen(seed, s2, s1, S2_dev, (cudaStream_t)stream);
  }));
  return RANDQR_OK;
}

randqr_status randqr_set_sketch_kind(randqr_ctx *ctx, int32_t kind) {
  if (!ctx || kind < RANDQR_SKETCH_GAUSSIAN || kind > RANDQR_SKETCH_GAUSSIAN_ONLY) return RANDQR_ERR_ARG;
  ctx->s2_kind = kind;
  return RANDQR_OK;
}

randqr_status randqr_sketch(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                            int64_t ldv, int64_t s1, int64_t s2, uint64_t seed,
                            const double *S2, double *Ws, void *stream) {
  if (!ctx || !V || !Ws || n < 1 || m < 1 || ldv < n || bad_sketch_sizes(n, s1, s2) ||
      bad_sketch_kind(ctx, m, s1, s2, 0))
    return RANDQR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  randqr_status st = begin_call(ctx, s);
  if (st != RANDQR_OK) return st;
  Workspace w;
  if ((st = carve(ctx, n, s1, s2, &w)) != RANDQR_OK) return st;
  if ((st = sketch_and_hhqr(ctx, V, m, n, ldv, s1, s2, seed, S2, w, s, false)) != RANDQR_OK)
    return st;
  RQ_CUDA(cudaMemcpyAsync(Ws, w.Ws, sizeof(double) * (size_t)(s2 * n), cudaMemcpyDeviceToDevice, s));
  return RANDQR_OK;
}

// Algorithm 3 from R_s on, with the row passes in pair arithmetic: W = V R_s^{-1} is kept
// in the Q buffer as (hi, lo) pairs, G = W^T W, R_c = chol(G) and R = R_c R_s in FP64, then
// Q = W R_c^{-1} written back as FP64 in place.
static randqr_status factor_df(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                               int64_t ldv, double *Q, int64_t ldq, double *R, int64_t ldr,
                               const Workspace &w, cudaStream_t s, randqr_info *info) {
  RQ_CUDA(timed(ctx, s, rq::K_PACK_DF, [&] { return rq::launch_pack_df(w.Rs, n, w.Rdf, w.rinv, ctx->status_dev, s); }));
  RQ_CUDA(timed(ctx, s, rq::K_TRSM_DF, [&] {
    return rq::launch_trsm_df(V, true, ldv, Q, false, ldq, m, n, w.Rdf, w.rinv, ctx->num_sms,
                              ctx->status_dev, s);
  }));
  RQ_CUDA(cudaMemsetAsync(w.G, 0, sizeof(double) * packed(n), s));
  if (ctx->use_tc && rq::gram_oz_supported(n)) {
    RQ_CUDA(timed(ctx, s, rq::K_GRAM_TC, [&] {
      return launch_gram_tc(ctx, Q, true, ldq, m, n, w.G, s);
    }));
  } else {
    RQ_CUDA(timed(ctx, s, rq::K_GRAM_DF, [&] {
      return rq::launch_gram_df((const float2 *)Q, ldq, m, n, w.G, ctx->num_sms, ctx->status_dev, s);
    }));
  }
  RQ_CUDA(timed(ctx, s, rq::K_POTRF, [&] {
    return rq::launch_potrf(w.G, n, 0.0, w.Rc, w.Rs, nullptr, R, ldr, 1, ctx->status_dev, s);
  }));
  RQ_CUDA(timed(ctx, s, rq::K_PACK_DF, [&] { return rq::launch_pack_df(w.Rc, n, w.Rdf, w.rinv, ctx->status_dev, s); }));
  RQ_CUDA(timed(ctx, s, rq::K_TRSM_DF, [&] {
    return rq::launch_trsm_df(Q, false, ldq, Q, true, ldq, m, n, w.Rdf, w.rinv, ctx->num_sms,
                              ctx->status_dev, s);
  }));
  return finish_call(ctx, s, info);
}

static randqr_status factor_impl(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                                 int64_t ldv, int64_t s1, int64_t s2, uint64_t seed,
                                 const double *S2, randqr_precision prec, double *Q, int64_t ldq,
                                 double *R, int64_t ldr, randqr_info *info, void *stream,
                                 bool second_pass) {
  if (!ctx || bad_factor_args(V, m, n, ldv, Q, ldq, R, ldr) || bad_sketch_sizes(n, s1, s2) ||
      bad_sketch_kind(ctx, m, s1, s2, 0) ||
      (prec != RANDQR_FP64 && prec != RANDQR_F32X2) || s2 > m)
    return RANDQR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  randqr_status st = begin_call(ctx, s);
  if (st != RANDQR_OK) return st;
  Workspace w;
  if ((st = carve(ctx, n, s1, s2, &w)) != RANDQR_OK) return st;
  if ((st = sketch_and_hhqr(ctx, V, m, n, ldv, s1, s2, seed, S2, w, s, true)) != RANDQR_OK)
    return st;
  if (second_pass && blocked_tc_ok(ctx, n, V, ldv, Q, ldq)) {
    // 64 < n <= 128: both solves blocked into split products (either precision)
    if ((st = blocked_first_solve_tc(ctx, V, ldv, Q, ldq, m, n, w.Rs, w, s)) != RANDQR_OK) return st;
    if ((st = cholqr_pass(ctx, Q, ldq, Q, ldq, m, n, 0.0, w.Rs, nullptr, R, ldr, 1, RANDQR_FP64, w, s,
                          /*inverse_ok=*/true)) != RANDQR_OK)
      return st;
    return finish_factor(ctx, s, info, V, ldv, Q, ldq, R, ldr, m, n);
  }
  if (second_pass && use_tc_solve(ctx, n)) {
    // Both solves as tensor-core products with explicit inverses: W = V (R_s^{-1}) into Q, then
    // the Cholesky pass on W in place.  RANDQR_F32X2 keeps six digits of the rows (46-bit
    // products, its stated precision) instead of seven.
    const int dg = prec == RANDQR_F32X2 ? 6 : 7;
    RQ_CUDA(timed(ctx, s, rq::K_TRI_INV, [&] { return rq::launch_tri_inv(w.Rs, n, w.Rt2, ctx->status_dev, s); }));
    // n = 64: the solve and the Gram of W in one launch (W stored once, its Gram taken on paired
    // CTAs as the rows are stored); otherwise the solve, then the Gram inside the Cholesky pass
    const bool fused = ctx->fuse_first_pass && rq::solve_gram_supported(n, V, ldv, Q, ldq, ctx->num_sms);
    if (fused) {
      RQ_CUDA(cudaMemsetAsync(w.G, 0, sizeof(double) * packed(n), s));
      RQ_CUDA(timed(ctx, s, rq::K_SOLVE_GRAM, [&] {
        return rq::launch_solve_gram(V, ldv, Q, ldq, m, n, w.Rt2, w.G, ctx->num_sms, ctx->status_dev, s, dg);
      }));
    } else {
      RQ_CUDA(timed(ctx, s, rq::K_TRSM_TC, [&] {
        return rq::launch_trsm_oz(V, ldv, Q, ldq, m, n, w.Rt2, ctx->num_sms, ctx->status_dev, s, dg);
      }));
    }
    if ((st = cholqr_pass(ctx, Q, ldq, Q, ldq, m, n, 0.0, w.Rs, nullptr, R, ldr, 1, RANDQR_FP64, w, s,
                          /*inverse_ok=*/true, dg, /*gram_done=*/fused)) != RANDQR_OK)
      return st;
    return finish_factor(ctx, s, info, V, ldv, Q, ldq, R, ldr, m, n);
  }
  if (prec == RANDQR_F32X2 && second_pass) {
    if ((st = factor_df(ctx, V, m, n, ldv, Q, ldq, R, ldr, w, s, nullptr)) != RANDQR_OK) return st;
    return finish_factor(ctx, s, info, V, ldv, Q, ldq, R, ldr, m, n);
  }
  if (!second_pass && (use_tc_solve(ctx, n) || blocked_tc_ok(ctx, n, V, ldv, Q, ldq))) {
    // randQR alone: Q = V R_s^{-1} by the same tensor-core solve as rand_cholQR's first pass
    if (n > 64) {
      if ((st = blocked_first_solve_tc(ctx, V, ldv, Q, ldq, m, n, w.Rs, w, s)) != RANDQR_OK) return st;
    } else {
      RQ_CUDA(timed(ctx, s, rq::K_TRI_INV, [&] { return rq::launch_tri_inv(w.Rs, n, w.Rt2, ctx->status_dev, s); }));
      RQ_CUDA(timed(ctx, s, rq::K_TRSM_TC, [&] {
        return rq::launch_trsm_oz(V, ldv, Q, ldq, m, n, w.Rt2, ctx->num_sms, ctx->status_dev, s);
      }));
    }
    RQ_CUDA(timed(ctx, s, rq::K_UNPACK, [&] { return rq::launch_unpack(w.Rs, n, R, ldr, ctx->status_dev, s); }));
    clear_accuracy(info);
    return finish_call(ctx, s, info);
  }
  // W = V R_s^{-1}, written into Q.
  RQ_CUDA(timed(ctx, s, rq::K_TRSM, [&] {
    return rq::launch_trsm(V, ldv, Q, ldq, m, n, w.Rs, RANDQR_FP64, ctx->num_sms, ctx->status_dev, s);
  }));
  if (!second_pass) {
    RQ_CUDA(timed(ctx, s, rq::K_UNPACK, [&] { return rq::launch_unpack(w.Rs, n, R, ldr, ctx->status_dev, s); }));
    clear_accuracy(info);
    return finish_call(ctx, s, info);
  }
  // cholQR of W, in place on Q; R = R_c R_s written dense.
  if ((st = cholqr_pass(ctx, Q, ldq, Q, ldq, m, n, 0.0, w.Rs, nullptr, R, ldr, 1, RANDQR_FP64, w, s,
                        /*inverse_ok=*/true)) != RANDQR_OK)
    return st;
  return finish_factor(ctx, s, info, V, ldv, Q, ldq, R, ldr, m, n);
}

randqr_status randqr_factor(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                            int64_t ldv, int64_t s1, int64_t s2, uint64_t seed,
                            const double *S2, randqr_precision prec, double *Q, int64_t ldq,
                            double *R, int64_t ldr, randqr_info *info, void *stream) {
  return factor_impl(ctx, V, m, n, ldv, s1, s2, seed, S2, prec, Q, ldq, R, ldr, info, stream,
                     true);
}

randqr_status randqr_factor_host(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                                 int64_t ldv, int64_t s1, int64_t s2, uint64_t seed,
                                 const double *S2, randqr_precision prec, double *Q, int64_t ldq,
                                 double *R, int64_t ldr, randqr_info *info, void *stream) {
  // the checks of randqr_factor before anything is staged
  if (!ctx || bad_factor_args(V, m, n, ldv, Q, ldq, R, ldr) ||
      ranges_overlap(R, span_bytes(n, n, ldr), V, span_bytes(m, n, ldv)) || bad_sketch_sizes(n, s1, s2) ||
      bad_sketch_kind(ctx, m, s1, s2, 0) || (prec != RANDQR_FP64 && prec != RANDQR_F32X2) || s2 > m)
    return RANDQR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  RQ_CUDA(cudaSetDevice(ctx->device));
  // V (packed to ld n) and R in the context's staging area; the factorization runs in place
  const size_t vbytes = align_up(sizeof(double) * (size_t)m * (size_t)n);
  randqr_status st = ensure_host_stage(ctx, vbytes + align_up(sizeof(double) * (size_t)(n * n)));
  if (st != RANDQR_OK) return st;
  double *Vd = (double *)ctx->hstage;
  double *Rd = (double *)((char *)ctx->hstage + vbytes);
  const size_t row = sizeof(double) * (size_t)n;
  RQ_CUDA(cudaMemcpy2DAsync(Vd, row, V, sizeof(double) * (size_t)ldv, row, (size_t)m, cudaMemcpyHostToDevice, s));
  st = factor_impl(ctx, Vd, m, n, n, s1, s2, seed, S2, prec, Vd, n, Rd, n, nullptr, stream, true);
  if (st != RANDQR_OK) return st;
  if (info && info->want_accuracy) {
    // the factorization ran in place on the staged V: only the orthogonality can be measured
    if ((st = rq_accuracy_enqueue(ctx, nullptr, 0, Vd, n, Rd, n, m, n, s)) != RANDQR_OK) return st;
  }
  RQ_CUDA(cudaMemcpy2DAsync(Q, sizeof(double) * (size_t)ldq, Vd, row, row, (size_t)m, cudaMemcpyDeviceToHost, s));
  RQ_CUDA(cudaMemcpy2DAsync(R, sizeof(double) * (size_t)ldr, Rd, row, row, (size_t)n, cudaMemcpyDeviceToHost, s));
  if (!info) return RANDQR_OK;
  const bool want = info->want_accuracy != 0;
  clear_accuracy(info);
  st = randqr_get_status(ctx, s, info);
  if (st == RANDQR_OK && want) rq_accuracy_finish(ctx, n, false, info);
  return st;
}

randqr_status randqr_randqr(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                            int64_t ldv, int64_t s1, int64_t s2, uint64_t seed,
                            const double *S2, double *Q0, int64_t ldq, double *R0,
                            int64_t ldr, randqr_info *info, void *stream) {
  return factor_impl(ctx, V, m, n, ldv, s1, s2, seed, S2, RANDQR_FP64, Q0, ldq, R0, ldr, info,
                     stream, false);
}

randqr_status randqr_cholqr2(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                             int64_t ldv, double *Q, int64_t ldq, double *R, int64_t ldr,
                             randqr_info *info, void *stream) {
  if (!ctx || bad_factor_args(V, m, n, ldv, Q, ldq, R, ldr)) return RANDQR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  randqr_status st = begin_call(ctx, s);
  if (st != RANDQR_OK) return st;
  Workspace w;
  if ((st = carve(ctx, n, 1, 1, &w)) != RANDQR_OK) return st;
  // pass 1: Q0 = V R0^{-1} into Q; keep R0 in w.Rt.  R0 is as ill conditioned as V (at most
  // about u^{-1/2} when the Cholesky factorization succeeds); a product with its computed
  // inverse X (R0 X = I + F, |F| <= gamma_n |R0| |X|) gives Q0 (I + F) with ||F|| of order
  // n u kappa(R0), far below pass 1's own loss of orthogonality (u kappa(V)^2), which pass 2
  // removes.  So both passes take the tensor-core products where they exist.
  if ((st = cholqr_pass(ctx, V, ldv, Q, ldq, m, n, 0.0, nullptr, nullptr, nullptr, 0, 1,
                        RANDQR_FP64, w, s, /*inverse_ok=*/true)) != RANDQR_OK)
    return st;
  RQ_CUDA(cudaMemcpyAsync(w.Rt, w.Rc, sizeof(double) * packed(n), cudaMemcpyDeviceToDevice, s));
  // pass 2 in place; R = R1 R0
  if ((st = cholqr_pass(ctx, Q, ldq, Q, ldq, m, n, 0.0, w.Rt, nullptr, R, ldr, 2, RANDQR_FP64,
                        w, s, /*inverse_ok=*/true)) != RANDQR_OK)
    return st;
  return finish_factor(ctx, s, info, V, ldv, Q, ldq, R, ldr, m, n);
}

randqr_status randqr_shifted_cholqr3(randqr_ctx *ctx, const double *V, int64_t m, int64_t n,
                                     int64_t ldv, double *Q, int64_t ldq, double *R,
                                     int64_t ldr, randqr_info *info, void *stream) {
  if (!ctx || bad_factor_args(V, m, n, ldv, Q, ldq, R, ldr)) return RANDQR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  randqr_status st = begin_call(ctx, s);
  if (st != RANDQR_OK) return st;
  Workspace w;
  if ((st = carve(ctx, n, 1, 1, &w)) != RANDQR_OK) return st;
  const double u = 1.1102230246251565404e-16;  // 2^-53
  const double coeff = 11.0 * ((double)m * (double)n + (double)n * (double)(n + 1)) * u;
  // shifted pass: R0 -> w.Rt.  The shift keeps kappa(R0) below about u^{-1/2}, so the solves
  // may run as products with computed inverses as in randqr_cholqr2.
  if ((st = cholqr_pass(ctx, V, ldv, Q, ldq, m, n, coeff, nullptr, nullptr, nullptr, 0, 1,
                        RANDQR_FP64, w, s, /*inverse_ok=*/true)) != RANDQR_OK)
    return st;
  RQ_CUDA(cudaMemcpyAsync(w.Rt, w.Rc, sizeof(double) * packed(n), cudaMemcpyDeviceToDevice, s));
  // cholQR2 of Q0: R1 R0 -> w.Rs (not used by this method otherwise; w.Rt2 holds the inverses
  // of the tensor-core solves), then R2 (R1 R0) dense
  if ((st = cholqr_pass(ctx, Q, ldq, Q, ldq, m, n, 0.0, w.Rt, w.Rs, nullptr, 0, 2, RANDQR_FP64,
                        w, s, /*inverse_ok=*/true)) != RANDQR_OK)
    return st;
  if ((st = cholqr_pass(ctx, Q, ldq, Q, ldq, m, n, 0.0, w.Rs, nullptr, R, ldr, 3, RANDQR_FP64,
                        w, s, /*inverse_ok=*/true)) != RANDQR_OK)
    return st;
  return finish_factor(ctx, s, info, V, ldv, Q, ldq, R, ldr, m, n);
}

// ---- Row-sharded rand_cholQR (Sec. 4.1): the stages between the two reductions ----------

randqr_status randqr_shard_sketch(randqr_ctx *ctx, const double *V, int64_t m, int64_t n, int64_t ldv,
                                  int64_t row0, int64_t s1, int64_t s2, uint64_t seed, const double *S2,
                                  double *Ws, void *stream) {
  if (!ctx || !V || !Ws || n < 1 || n > kMaxN || m < 1 || ldv < n || row0 < 0 ||
      bad_sketch_sizes(n, s1, s2) || bad_sketch_kind(ctx, m, s1, s2, row0) ||
      ctx->s2_kind == RANDQR_SKETCH_GAUSSIAN_ONLY)
    return RANDQR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  randqr_status st = begin_call(ctx, s);
  if (st != RANDQR_OK) return st;
  Workspace w;
  if ((st = carve(ctx, n, s1, s2, &w)) != RANDQR_OK) return st;
  if ((st = sketch_and_hhqr(ctx, V, m, n, ldv, s1, s2, seed, S2, w, s, false, row0)) != RANDQR_OK)
    return st;
  RQ_CUDA(cudaMemcpyAsync(Ws, w.Ws, sizeof(double) * (size_t)(s2 * n), cudaMemcpyDeviceToDevice, s));
  return RANDQR_OK;
}

randqr_status randqr_sketch_r(randqr_ctx *ctx, const double *Ws, int64_t s2, int64_t n, double *Rs,
                              int64_t ldr, randqr_info *info, void *stream) {
  if (!ctx || !Ws || !Rs || n < 1 || n > kMaxN || s2 < n || s2 > ((int64_t)1 << 20) || ldr < n)
    return RANDQR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  randqr_status st = begin_call(ctx, s);
  if (st != RANDQR_OK) return st;
  Workspace w;
  if ((st = carve(ctx, n, s2, s2, &w)) != RANDQR_OK) return st;
  RQ_CUDA(cudaMemcpyAsync(w.Ws, Ws, sizeof(double) * (size_t)(s2 * n), cudaMemcpyDeviceToDevice, s));
  RQ_CUDA(timed(ctx, s, rq::K_HHQR, [&] { return rq::launch_hhqr(w.Ws, s2, n, w.Rs, w.hq, ctx->status_dev, s); }));
  RQ_CUDA(timed(ctx, s, rq::K_UNPACK, [&] { return rq::launch_unpack(w.Rs, n, Rs, ldr, ctx->status_dev, s); }));
  return finish_call(ctx, s, info);
}

randqr_status randqr_shard_gram(randqr_ctx *ctx, const double *V, int64_t m, int64_t n, int64_t ldv,
                                const double *Rs, int64_t ldrs, double *Q, int64_t ldq, double *G,
                                int64_t ldg, void *stream) {
  if (!ctx || !Rs || !G || ldrs < n || ldg < n || bad_factor_args(V, m, n, ldv, Q, ldq, G, ldg, true))
    return RANDQR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  randqr_status st = begin_call(ctx, s);
  if (st != RANDQR_OK) return st;
  Workspace w;
  if ((st = carve(ctx, n, 1, 1, &w)) != RANDQR_OK) return st;
  RQ_CUDA(timed(ctx, s, rq::K_UNPACK, [&] { return rq::launch_pack_upper(Rs, ldrs, n, w.Rs, ctx->status_dev, s); }));
  // W_k = V_k R_s^{-1} into Q (as in randqr_factor), then G_k = W_k^T W_k: one fused launch
  // where randqr_factor takes it, else the solve and then the Gram
  const bool fused = use_tc_solve(ctx, n) && ctx->fuse_first_pass &&
                     rq::solve_gram_supported(n, V, ldv, Q, ldq, ctx->num_sms);
  if (fused) {
    RQ_CUDA(timed(ctx, s, rq::K_TRI_INV, [&] { return rq::launch_tri_inv(w.Rs, n, w.Rt2, ctx->status_dev, s); }));
    RQ_CUDA(cudaMemsetAsync(w.G, 0, sizeof(double) * packed(n), s));
    RQ_CUDA(timed(ctx, s, rq::K_SOLVE_GRAM, [&] {
      return rq::launch_solve_gram(V, ldv, Q, ldq, m, n, w.Rt2, w.G, ctx->num_sms, ctx->status_dev, s, 7);
    }));
  } else if (use_tc_solve(ctx, n)) {
    RQ_CUDA(timed(ctx, s, rq::K_TRI_INV, [&] { return rq::launch_tri_inv(w.Rs, n, w.Rt2, ctx->status_dev, s); }));
    RQ_CUDA(timed(ctx, s, rq::K_TRSM_TC, [&] {
      return rq::launch_trsm_oz(V, ldv, Q, ldq, m, n, w.Rt2, ctx->num_sms, ctx->status_dev, s);
    }));
  } else {
    RQ_CUDA(timed(ctx, s, rq::K_TRSM, [&] {
      return rq::launch_trsm(V, ldv, Q, ldq, m, n, w.Rs, RANDQR_FP64, ctx->num_sms, ctx->status_dev, s);
    }));
  }
  if (!fused) {
    RQ_CUDA(cudaMemsetAsync(w.G, 0, sizeof(double) * packed(n), s));
    if (ctx->use_tc && rq::gram_oz_supported(n)) {
      RQ_CUDA(timed(ctx, s, rq::K_GRAM_TC, [&] { return launch_gram_tc(ctx, Q, false, ldq, m, n, w.G, s); }));
    } else {
      RQ_CUDA(timed(ctx, s, rq::K_GRAM, [&] {
        return rq::launch_gram(Q, ldq, m, n, w.G, RANDQR_FP64, ctx->num_sms, ctx->status_dev, s);
      }));
    }
  }
  RQ_CUDA(timed(ctx, s, rq::K_UNPACK, [&] { return rq::launch_unpack_sym(w.G, n, G, ldg, ctx->status_dev, s); }));
  return RANDQR_OK;
}

randqr_status randqr_shard_finish(randqr_ctx *ctx, double *Q, int64_t m, int64_t n, int64_t ldq,
                                  const double *G, int64_t ldg, const double *Rs, int64_t ldrs, double *R,
                                  int64_t ldr, randqr_info *info, void *stream) {
  if (!ctx || !G || !Rs || ldg < n || ldrs < n || bad_factor_args(Q, m, n, ldq, Q, ldq, R, ldr, true))
    return RANDQR_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  randqr_status st = begin_call(ctx, s);
  if (st != RANDQR_OK) return st;
  Workspace w;
  if ((st = carve(ctx, n, 1, 1, &w)) != RANDQR_OK) return st;
  RQ_CUDA(timed(ctx, s, rq::K_UNPACK, [&] { return rq::launch_pack_upper(Rs, ldrs, n, w.Rs, ctx->status_dev, s); }));
  RQ_CUDA(timed(ctx, s, rq::K_UNPACK, [&] { return rq::launch_pack_upper(G, ldg, n, w.G, ctx->status_dev, s); }));
  RQ_CUDA(timed(ctx, s, rq::K_POTRF, [&] {
    return rq::launch_potrf(w.G, n, 0.0, w.Rc, w.Rs, nullptr, R, ldr, 1, ctx->status_dev, s);
  }));
  if (use_tc_solve(ctx, n)) {
    if ((st = solve_by_inverse_tc(ctx, Q, ldq, Q, ldq, m, n, w, s)) != RANDQR_OK) return st;
  } else {
    RQ_CUDA(timed(ctx, s, rq::K_TRSM, [&] {
      return rq::launch_trsm(Q, ldq, Q, ldq, m, n, w.Rc, RANDQR_FP64, ctx->num_sms, ctx->status_dev, s);
    }));
  }
  return finish_call(ctx, s, info);
}

}  // extern "C"
