// batch.cu -- randqr_factor_batched: many independent rand_cholQR factorizations of uneven
// sizes as one CUDA graph.
//
// A plan assigns the matrices to L "lanes" (streams, each with its own workspace context)
// and captures every lane's kernel chain -- sketch, Householder R_s, the row passes,
// Cholesky, the status copy -- as parallel branches of one graph, so small and large
// factorizations overlap on the device and the whole batch costs one graph launch.  The
// first call with a given batch (same descriptors, same precision) builds the plan: it
// warms every lane's workspace with uncaptured runs, then an autotuner captures candidate
// schedules (lane counts 4..32, items dealt to lanes largest-first) and keeps the fastest
// by timing graph replays.  Later calls with the same batch replay the kept graph.
// The paper factors one matrix at a time; batching is this library's addition.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <numeric>
#include <tuple>

#include "common.cuh"

namespace {

struct Plan {
  int lanes = 0;
  std::vector<randqr_ctx *> subs;
  std::vector<cudaStream_t> streams;
  cudaGraphExec_t exec = nullptr;
  rq::DevStatus *st_dev = nullptr;   // one status record per item
  rq::DevStatus *st_host = nullptr;  // pinned copy
  int count = 0;
  float best_ms = 0.f;
};

void destroy_plan(Plan *p) {
  if (!p) return;
  for (cudaStream_t s : p->streams) cudaStreamSynchronize(s);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  for (randqr_ctx *c : p->subs) randqr_destroy(c);
  for (cudaStream_t s : p->streams) cudaStreamDestroy(s);
  if (p->st_dev) cudaFree(p->st_dev);
  if (p->st_host) cudaFreeHost(p->st_host);
  delete p;
}

uint64_t fnv1a(const void *data, size_t len, uint64_t h) {
  const unsigned char *b = (const unsigned char *)data;
  for (size_t i = 0; i < len; ++i) {
    h ^= b[i];
    h *= 0x100000001b3ULL;
  }
  return h;
}

void sizes_of(const randqr_batch_item &it, int64_t *s1, int64_t *s2) {
  *s1 = it.s1 > 0 ? it.s1 : 2 * (it.n * it.n + it.n);
  *s2 = it.s2 > 0 ? it.s2 : 4 * it.n;
}

bool bad_item(const randqr_batch_item &it) {
  int64_t s1, s2;
  sizes_of(it, &s1, &s2);
  return !it.V || !it.Q || !it.R || it.n < 1 || it.n > 128 || it.m < it.n || it.ldv < it.n ||
         it.ldq < it.n || it.ldr < it.n || s2 < it.n || s1 < s2 || s2 > it.m ||
         s1 >= ((int64_t)1 << 31);
}

}  // namespace

struct randqr_batcher {
  std::map<uint64_t, Plan *> plans;
  std::map<std::tuple<uint64_t, int64_t, int64_t>, double *> s2_cache;
  cudaStream_t aux = nullptr;
};

void rq_batcher_destroy(randqr_ctx *ctx) {
  randqr_batcher *b = ctx->batcher;
  if (!b) return;
  cudaSetDevice(ctx->device);
  for (auto &kv : b->plans) destroy_plan(kv.second);
  for (auto &kv : b->s2_cache) cudaFree(kv.second);
  if (b->aux) cudaStreamDestroy(b->aux);
  delete b;
  ctx->batcher = nullptr;
}

namespace {

randqr_status s2_for(randqr_ctx *ctx, randqr_batcher *b, uint64_t seed, int64_t s1, int64_t s2,
                     const double **out) {
  auto key = std::make_tuple(seed, s1, s2);
  auto it = b->s2_cache.find(key);
  if (it != b->s2_cache.end()) {
    *out = it->second;
    return RANDQR_OK;
  }
  double *p = nullptr;
  if (cudaMalloc(&p, sizeof(double) * (size_t)(s1 * s2)) != cudaSuccess) {
    cudaGetLastError();
    return RANDQR_ERR_NOMEM;
  }
  if (randqr_gauss_sketch(ctx, seed, s2, s1, p, b->aux) != RANDQR_OK ||
      cudaStreamSynchronize(b->aux) != cudaSuccess) {
    cudaFree(p);
    return RANDQR_ERR_CUDA;
  }
  b->s2_cache[key] = p;
  *out = p;
  return RANDQR_OK;
}

// Enqueue item i on lane l of plan p (used both uncaptured, to size the lane's workspace,
// and under capture); the item's status record is copied out at the end of its chain.
randqr_status enqueue_item(Plan *p, int l, int i, const randqr_batch_item &it, const double *S2,
                           randqr_precision prec) {
  int64_t s1, s2;
  sizes_of(it, &s1, &s2);
  randqr_status st = randqr_factor(p->subs[l], it.V, it.m, it.n, it.ldv, s1, s2, it.seed, S2, prec,
                                   it.Q, it.ldq, it.R, it.ldr, nullptr, p->streams[l]);
  if (st != RANDQR_OK) return st;
  if (cudaMemcpyAsync(p->st_dev + i, p->subs[l]->status_dev, sizeof(rq::DevStatus),
                      cudaMemcpyDeviceToDevice, p->streams[l]) != cudaSuccess)
    return RANDQR_ERR_CUDA;
  return RANDQR_OK;
}

// Build a plan with L lanes; items dealt largest-first round-robin.
randqr_status build_plan(randqr_ctx *ctx, const randqr_batch_item *items,
                         int count, randqr_precision prec, const std::vector<const double *> &s2p,
                         int L, cudaStream_t timing_stream, Plan **out) {
  Plan *p = new (std::nothrow) Plan();
  if (!p) return RANDQR_ERR_NOMEM;
  p->lanes = L;
  p->count = count;
  randqr_status st = RANDQR_OK;
  if (cudaMalloc(&p->st_dev, sizeof(rq::DevStatus) * count) != cudaSuccess ||
      cudaMallocHost(&p->st_host, sizeof(rq::DevStatus) * count) != cudaSuccess) {
    cudaGetLastError();
    destroy_plan(p);
    return RANDQR_ERR_NOMEM;
  }
  for (int l = 0; l < L; ++l) {
    cudaStream_t s = nullptr;
    randqr_ctx *c = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        randqr_create(&c, ctx->device, 0) != RANDQR_OK) {
      cudaGetLastError();
      if (s) cudaStreamDestroy(s);
      destroy_plan(p);
      return RANDQR_ERR_CUDA;
    }
    rq_inherit_settings(c, ctx);
    p->streams.push_back(s);
    p->subs.push_back(c);
  }
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    return items[a].m * items[a].n * items[a].n > items[c].m * items[c].n * items[c].n;
  });
  std::vector<int> lane_of(count);
  for (int k = 0; k < count; ++k) lane_of[order[k]] = k % L;
  // warm-up: size every lane's workspace outside capture
  for (int k = 0; k < count && st == RANDQR_OK; ++k) {
    const int i = order[k];
    st = enqueue_item(p, lane_of[i], i, items[i], s2p[i], prec);
  }
  for (cudaStream_t s : p->streams)
    if (cudaStreamSynchronize(s) != cudaSuccess) st = RANDQR_ERR_CUDA;
  if (st != RANDQR_OK) {
    destroy_plan(p);
    return st;
  }
  // capture: fork from an origin stream into the lanes, join back
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins(L, nullptr);
  cudaGraph_t graph = nullptr;
  bool ok = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
  for (int l = 0; ok && l < L; ++l)
    ok = cudaEventCreateWithFlags(&joins[l], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) == cudaSuccess &&
       cudaEventRecord(fork, origin) == cudaSuccess;
  for (int l = 0; ok && l < L; ++l) ok = cudaStreamWaitEvent(p->streams[l], fork, 0) == cudaSuccess;
  for (int k = 0; ok && k < count; ++k) {
    const int i = order[k];
    ok = enqueue_item(p, lane_of[i], i, items[i], s2p[i], prec) == RANDQR_OK;
  }
  for (int l = 0; ok && l < L; ++l)
    ok = cudaEventRecord(joins[l], p->streams[l]) == cudaSuccess &&
         cudaStreamWaitEvent(origin, joins[l], 0) == cudaSuccess;
  cudaError_t ec = cudaStreamEndCapture(origin, &graph);
  ok = ok && ec == cudaSuccess && graph;
  ok = ok && cudaGraphInstantiate(&p->exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  // time two replays
  if (ok) {
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    ok = cudaEventCreate(&t0) == cudaSuccess && cudaEventCreate(&t1) == cudaSuccess &&
         cudaGraphLaunch(p->exec, timing_stream) == cudaSuccess &&
         cudaEventRecord(t0, timing_stream) == cudaSuccess &&
         cudaGraphLaunch(p->exec, timing_stream) == cudaSuccess &&
         cudaGraphLaunch(p->exec, timing_stream) == cudaSuccess &&
         cudaEventRecord(t1, timing_stream) == cudaSuccess &&
         cudaEventSynchronize(t1) == cudaSuccess &&
         cudaEventElapsedTime(&p->best_ms, t0, t1) == cudaSuccess;
    p->best_ms *= 0.5f;
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
  }
  for (cudaEvent_t e : joins)
    if (e) cudaEventDestroy(e);
  if (fork) cudaEventDestroy(fork);
  if (origin) cudaStreamDestroy(origin);
  if (!ok) {
    cudaGetLastError();
    destroy_plan(p);
    return RANDQR_ERR_CUDA;
  }
  *out = p;
  return RANDQR_OK;
}

}  // namespace

extern "C" randqr_status randqr_factor_batched(randqr_ctx *ctx, const randqr_batch_item *items,
                                               int32_t count, randqr_precision prec,
                                               randqr_status *statuses, void *stream) {
  if (!ctx || count < 0 || (count > 0 && !items) ||
      (prec != RANDQR_FP64 && prec != RANDQR_F32X2))
    return RANDQR_ERR_ARG;
  if (count == 0) return RANDQR_OK;
  for (int32_t i = 0; i < count; ++i)
    if (bad_item(items[i])) return RANDQR_ERR_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return RANDQR_ERR_CUDA;
  if (!ctx->batcher) {
    ctx->batcher = new (std::nothrow) randqr_batcher();
    if (!ctx->batcher) return RANDQR_ERR_NOMEM;
    if (cudaStreamCreateWithFlags(&ctx->batcher->aux, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx->batcher;
      ctx->batcher = nullptr;
      return RANDQR_ERR_CUDA;
    }
  }
  randqr_batcher *b = ctx->batcher;
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t key = fnv1a(items, sizeof(randqr_batch_item) * (size_t)count, 0xcbf29ce484222325ULL);
  key = fnv1a(&prec, sizeof(prec), key);
  Plan *plan = nullptr;
  auto found = b->plans.find(key);
  if (found != b->plans.end()) {
    plan = found->second;
  } else {
    std::vector<const double *> s2p(count);
    for (int32_t i = 0; i < count; ++i) {
      int64_t s1, s2;
      sizes_of(items[i], &s1, &s2);
      randqr_status st = s2_for(ctx, b, items[i].seed + 1, s1, s2, &s2p[i]);
      if (st != RANDQR_OK) return st;
    }
    // autotune the lane count on this batch
    const int cand[] = {4, 8, 16, 32};
    for (int L : cand) {
      if (L > count && L != cand[0]) break;
      Plan *p = nullptr;
      randqr_status st = build_plan(ctx, items, count, prec, s2p, std::min<int>(L, count), s, &p);
      if (st != RANDQR_OK) {
        destroy_plan(plan);
        return st;
      }
      if (!plan || p->best_ms < plan->best_ms) {
        destroy_plan(plan);
        plan = p;
      } else {
        destroy_plan(p);
      }
    }
    b->plans[key] = plan;
  }
  if (cudaGraphLaunch(plan->exec, s) != cudaSuccess) {
    cudaGetLastError();
    return RANDQR_ERR_CUDA;
  }
  if (!statuses) return RANDQR_OK;
  if (cudaMemcpyAsync(plan->st_host, plan->st_dev, sizeof(rq::DevStatus) * count,
                      cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return RANDQR_ERR_CUDA;
  }
  randqr_status first = RANDQR_OK;
  for (int32_t i = 0; i < count; ++i) {
    statuses[i] = (randqr_status)plan->st_host[i].code;
    if (first == RANDQR_OK && statuses[i] != RANDQR_OK) first = statuses[i];
  }
  return first;
}

extern "C" randqr_status randqr_batch_plan_info(randqr_ctx *ctx, const randqr_batch_item *items,
                                                int32_t count, randqr_precision prec,
                                                int32_t *lanes, float *ms) {
  if (!ctx || !items || count < 1) return RANDQR_ERR_ARG;
  if (!ctx->batcher) return RANDQR_ERR_TICKET;
  uint64_t key = fnv1a(items, sizeof(randqr_batch_item) * (size_t)count, 0xcbf29ce484222325ULL);
  key = fnv1a(&prec, sizeof(prec), key);
  auto it = ctx->batcher->plans.find(key);
  if (it == ctx->batcher->plans.end()) return RANDQR_ERR_TICKET;
  if (lanes) *lanes = it->second->lanes;
  if (ms) *ms = it->second->best_ms;
  return RANDQR_OK;
}
