// serve.cu -- randqr_submit / randqr_poll: continuous batching of factorization requests.
//
// The server of a context owns S "slots".  Each slot is a CUDA stream with its own
// sub-context (workspace and device status word), so requests in different slots run
// concurrently on the device.  Requests wait in a FIFO queue and are admitted, in order, as
// soon as a slot is free and their footprint fits the HBM budget next to everything in
// flight; completion is observed through an event recorded after the status word's copy
// to pinned host memory, so polling never blocks and a finished slot is refilled at once.
// The Gaussian sketches S2 are generated once per (seed, s1, s2) and shared by all slots.
// The paper has no serving layer; this is the request path around its Algorithms 3-4.
#include <stdio.h>

#include <chrono>
#include <deque>
#include <map>
#include <tuple>
#include <unordered_map>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { QUEUED = 0, RUNNING = 1, DONE = 2 };

struct Req {
  randqr_request r;
  size_t bytes = 0;
  int slot = -1;
  ReqState state = QUEUED;
  randqr_status status = RANDQR_PENDING;
  randqr_info info{};
  int used_prec = RANDQR_FP64;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  randqr_ctx *sub = nullptr;
  uint64_t ticket = 0;
  bool busy = false;
};

}  // namespace

struct randqr_server {
  int device = 0;
  size_t budget = 0;
  size_t in_flight = 0;
  uint64_t next_ticket = 1;
  uint64_t submitted = 0, completed = 0;
  std::vector<Slot> slots;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  std::map<std::tuple<uint64_t, int64_t, int64_t>, double *> s2_cache;
  size_t s2_bytes = 0;
  cudaStream_t aux = nullptr;
};

namespace {

constexpr int kDefaultSlots = 8;
constexpr size_t kDefaultBudget = (size_t)64 << 30;

void sketch_sizes(const randqr_request &r, int64_t *s1, int64_t *s2) {
  *s1 = r.s1 > 0 ? r.s1 : 2 * (r.n * r.n + r.n);
  *s2 = r.s2 > 0 ? r.s2 : 4 * r.n;
}

// Device bytes a request holds while in flight: its V, Q, R and the slot workspace it needs.
size_t footprint(const randqr_request &r) {
  int64_t s1, s2;
  sketch_sizes(r, &s1, &s2);
  size_t b = sizeof(double) * (size_t)(r.m * r.ldv + r.m * r.ldq + r.n * r.ldr);
  if (r.algo == RANDQR_ALGO_RAND_CHOLQR) b += sizeof(double) * (size_t)(s1 * r.n + s2 * r.n);
  b += sizeof(double) * (size_t)(8 * r.n * r.n);
  return b;
}

bool bad_request(const randqr_request &r) {
  if (r.algo < RANDQR_ALGO_RAND_CHOLQR || r.algo > RANDQR_ALGO_SHIFTED_CHOLQR3) return true;
  if (r.prec != RANDQR_FP64 && r.prec != RANDQR_F32X2) return true;
  if (r.reserved != 0) return true;  // a descriptor written by a different build, or corrupted
  if (rq::factor_args_bad(r.V, r.m, r.n, r.ldv, r.Q, r.ldq, r.R, r.ldr)) return true;
  if (r.algo == RANDQR_ALGO_RAND_CHOLQR) {
    int64_t s1, s2;
    sketch_sizes(r, &s1, &s2);
    if (s2 < r.n || s1 < s2 || s2 > r.m || s1 >= ((int64_t)1 << 31)) return true;
  }
  return false;
}

randqr_status server_init(randqr_ctx *ctx, int slots, size_t budget) {
  randqr_server *sv = new (std::nothrow) randqr_server();
  if (!sv) return RANDQR_ERR_NOMEM;
  sv->device = ctx->device;
  sv->budget = budget ? budget : kDefaultBudget;
  if (cudaSetDevice(ctx->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&sv->aux, cudaStreamNonBlocking) != cudaSuccess) {
    delete sv;
    return RANDQR_ERR_CUDA;
  }
  sv->slots.resize(slots);
  for (auto &sl : sv->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
        randqr_create(&sl.sub, ctx->device, 0) != RANDQR_OK) {
      ctx->server = sv;
      rq_server_destroy(ctx);
      return RANDQR_ERR_CUDA;
    }
  }
  ctx->server = sv;
  return RANDQR_OK;
}

// S2 for (seed, s1, s2): generated once on the aux stream, waited for, then shared.
randqr_status cached_s2(randqr_ctx *ctx, randqr_server *sv, uint64_t seed, int64_t s1,
                        int64_t s2, const double **out) {
  auto key = std::make_tuple(seed, s1, s2);
  auto it = sv->s2_cache.find(key);
  if (it != sv->s2_cache.end()) {
    *out = it->second;
    return RANDQR_OK;
  }
  double *p = nullptr;
  const size_t bytes = sizeof(double) * (size_t)(s1 * s2);
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return RANDQR_ERR_NOMEM;
  }
  if (randqr_gauss_sketch(ctx, seed, s2, s1, p, sv->aux) != RANDQR_OK ||
      cudaStreamSynchronize(sv->aux) != cudaSuccess) {
    cudaFree(p);
    return RANDQR_ERR_CUDA;
  }
  sv->s2_cache[key] = p;
  sv->s2_bytes += bytes;
  *out = p;
  return RANDQR_OK;
}

// Enqueue request t on slot i.
randqr_status start(randqr_ctx *ctx, randqr_server *sv, uint64_t t, int i) {
  Req &q = sv->reqs[t];
  Slot &sl = sv->slots[i];
  const randqr_request &r = q.r;
  randqr_status st;
  if (r.algo == RANDQR_ALGO_RAND_CHOLQR) {
    int64_t s1, s2;
    sketch_sizes(r, &s1, &s2);
    const double *S2 = nullptr;
    if ((st = cached_s2(ctx, sv, r.seed + 1, s1, s2, &S2)) != RANDQR_OK) return st;
    // the caller accepts 1e-12 or worse: the pair-arithmetic row passes meet that bound
    int prec = r.prec;
    if (prec == RANDQR_FP64 && r.max_orth_err >= 1e-12) prec = RANDQR_F32X2;
    q.used_prec = prec;
    rq_inherit_settings(sl.sub, ctx);
    st = randqr_factor(sl.sub, r.V, r.m, r.n, r.ldv, s1, s2, r.seed, S2, (randqr_precision)prec,
                       r.Q, r.ldq, r.R, r.ldr, nullptr, sl.stream);
  } else if (r.algo == RANDQR_ALGO_CHOLQR2) {
    rq_inherit_settings(sl.sub, ctx);
    st = randqr_cholqr2(sl.sub, r.V, r.m, r.n, r.ldv, r.Q, r.ldq, r.R, r.ldr, nullptr, sl.stream);
  } else {
    rq_inherit_settings(sl.sub, ctx);
    st = randqr_shifted_cholqr3(sl.sub, r.V, r.m, r.n, r.ldv, r.Q, r.ldq, r.R, r.ldr, nullptr,
                                sl.stream);
  }
  if (st != RANDQR_OK) return st;
  if (r.want_accuracy &&
      (st = rq_accuracy_enqueue(sl.sub, r.V, r.ldv, r.Q, r.ldq, r.R, r.ldr, r.m, r.n, sl.stream)) != RANDQR_OK)
    return st;
  if (cudaMemcpyAsync(sl.sub->status_host, sl.sub->status_dev, sizeof(rq::DevStatus),
                      cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
      cudaEventRecord(sl.done, sl.stream) != cudaSuccess)
    return RANDQR_ERR_CUDA;
  sl.busy = true;
  sl.ticket = t;
  q.slot = i;
  q.state = RUNNING;
  sv->in_flight += q.bytes;
  return RANDQR_OK;
}

// Retire finished slots, then admit queued requests in FIFO order while slots and memory
// allow.  Never blocks.
randqr_status pump(randqr_ctx *ctx, randqr_server *sv) {
  for (int i = 0; i < (int)sv->slots.size(); ++i) {
    Slot &sl = sv->slots[i];
    if (!sl.busy) continue;
    cudaError_t e = cudaEventQuery(sl.done);
    if (e == cudaErrorNotReady) continue;
    Req &q = sv->reqs[sl.ticket];
    if (e != cudaSuccess) {
      cudaGetLastError();
      q.status = RANDQR_ERR_CUDA;
    } else {
      const rq::DevStatus h = *sl.sub->status_host;
      q.status = (randqr_status)h.code;
      q.info.info = h.info;
      q.info.stage = h.stage;
      q.info.rs_min_diag = h.dmin;
      q.info.rs_max_diag = h.dmax;
      q.info.want_accuracy = q.r.want_accuracy;
      q.info.orth_err2 = -1.0;
      q.info.resid_relF = -1.0;
      if (q.status == RANDQR_OK && q.r.want_accuracy)
        rq_accuracy_finish(sl.sub, q.r.n, rq_accuracy_has_resid(q.r.V, q.r.Q), &q.info);
    }
    q.state = DONE;
    q.slot = -1;
    sv->in_flight -= q.bytes;
    sv->completed++;
    sl.busy = false;
  }
  while (!sv->queue.empty()) {
    int free_slot = -1;
    for (int i = 0; i < (int)sv->slots.size(); ++i)
      if (!sv->slots[i].busy) { free_slot = i; break; }
    if (free_slot < 0) break;
    const uint64_t t = sv->queue.front();
    if (sv->in_flight > 0 && sv->in_flight + sv->reqs[t].bytes > sv->budget) break;
    sv->queue.pop_front();
    randqr_status st = start(ctx, sv, t, free_slot);
    if (st != RANDQR_OK) {
      Req &q = sv->reqs[t];
      q.state = DONE;
      q.status = st;
      sv->completed++;
    }
  }
  return RANDQR_OK;
}

randqr_status get_server(randqr_ctx *ctx, randqr_server **out) {
  if (!ctx->server) {
    randqr_status st = server_init(ctx, kDefaultSlots, ctx->budget);
    if (st != RANDQR_OK) return st;
  }
  *out = ctx->server;
  return RANDQR_OK;
}

}  // namespace

void rq_server_destroy(randqr_ctx *ctx) {
  randqr_server *sv = ctx->server;
  if (!sv) return;
  cudaSetDevice(sv->device);
  for (auto &sl : sv->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.sub) randqr_destroy(sl.sub);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  for (auto &kv : sv->s2_cache) cudaFree(kv.second);
  if (sv->aux) cudaStreamDestroy(sv->aux);
  delete sv;
  ctx->server = nullptr;
}

extern "C" {

randqr_status randqr_serve_config(randqr_ctx *ctx, int32_t slots, size_t hbm_budget_bytes) {
  if (!ctx || slots < 1 || slots > 256) return RANDQR_ERR_ARG;
  if (ctx->server) {
    if (!ctx->server->queue.empty() || ctx->server->in_flight) return RANDQR_ERR_ARG;
    rq_server_destroy(ctx);
  }
  return server_init(ctx, slots, hbm_budget_bytes);
}

randqr_status randqr_submit(randqr_ctx *ctx, const randqr_request *req, uint64_t *ticket) {
  if (!ctx || !req || !ticket || bad_request(*req)) return RANDQR_ERR_ARG;
  randqr_server *sv;
  randqr_status st = get_server(ctx, &sv);
  if (st != RANDQR_OK) return st;
  Req q;
  q.r = *req;
  q.bytes = footprint(*req);
  if (q.bytes > sv->budget) return RANDQR_ERR_ADMISSION;
  const uint64_t t = sv->next_ticket++;
  sv->reqs.emplace(t, q);
  sv->queue.push_back(t);
  sv->submitted++;
  *ticket = t;
  return pump(ctx, sv);
}

randqr_status randqr_submit_batch(randqr_ctx *ctx, const randqr_request *reqs, int32_t count,
                                  uint64_t *tickets) {
  if (!ctx || count < 0 || (count > 0 && (!reqs || !tickets))) return RANDQR_ERR_ARG;
  for (int32_t i = 0; i < count; ++i)
    if (bad_request(reqs[i])) return RANDQR_ERR_ARG;
  for (int32_t i = 0; i < count; ++i) {
    randqr_status st = randqr_submit(ctx, &reqs[i], &tickets[i]);
    if (st != RANDQR_OK) return st;
  }
  return RANDQR_OK;
}

randqr_status randqr_poll(randqr_ctx *ctx, uint64_t ticket, randqr_info *info) {
  if (!ctx) return RANDQR_ERR_ARG;
  randqr_server *sv = ctx->server;
  if (!sv) return RANDQR_ERR_TICKET;
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return RANDQR_ERR_TICKET;
  pump(ctx, sv);
  Req &q = it->second;
  if (q.state != DONE) return RANDQR_PENDING;
  const randqr_status st = q.status;
  if (info) *info = q.info;
  sv->reqs.erase(it);
  return st;
}

randqr_status randqr_wait(randqr_ctx *ctx, uint64_t ticket, randqr_info *info) {
  if (!ctx) return RANDQR_ERR_ARG;
  for (;;) {
    randqr_status st = randqr_poll(ctx, ticket, info);
    if (st != RANDQR_PENDING) return st;
    randqr_server *sv = ctx->server;
    const Req &q = sv->reqs[ticket];
    if (q.state == RUNNING) {
      cudaEventSynchronize(sv->slots[q.slot].done);
    } else {  // queued: wait for any running slot to finish
      for (auto &sl : sv->slots)
        if (sl.busy) { cudaEventSynchronize(sl.done); break; }
    }
  }
}

randqr_status randqr_serve_stats_get(randqr_ctx *ctx, randqr_serve_stats *out) {
  if (!ctx || !out) return RANDQR_ERR_ARG;
  randqr_server *sv = ctx->server;
  *out = randqr_serve_stats{};
  if (!sv) return RANDQR_OK;
  pump(ctx, sv);
  out->submitted = sv->submitted;
  out->completed = sv->completed;
  out->queued = sv->queue.size();
  uint64_t running = 0;
  for (auto &sl : sv->slots) running += sl.busy;
  out->running = running;
  out->bytes_in_flight = sv->in_flight;
  out->slots = (int32_t)sv->slots.size();
  out->budget = sv->budget;
  return RANDQR_OK;
}

}  // extern "C"
