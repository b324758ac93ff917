// sketch_static.cu -- randqr_sketch_static: the multisketch Ws = S2 S1 V with its scratch
// in a fixed device array instead of context-owned memory, for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a sketch: code running
// inside a framework that owns every device allocation through its own pool, code called
// from a host callback or a real-time path where a blocking allocation (which may
// synchronise the device) is not allowed, or a library that must not grow the process's
// footprint behind its host application's back.  This entry point needs no context (whose
// creation allocates) and performs no allocation: the CountSketch accumulator W1 and the
// device status word live in the file-scope arrays below, which every GPU that loads the
// library holds until the process exits (8 MiB + 64 bytes per device).
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int64_t kStaticW1Max = int64_t(1) << 20;  // doubles: s1 * n <= 1,048,576 (8 MiB)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_w1[kStaticW1Max];
static __device__ __align__(256) rq::DevStatus g_static_status;

struct StaticSlot {
  bool ready = false;
  double *w1 = nullptr;
  rq::DevStatus *status = nullptr;
  int num_sms = 0;
};

StaticSlot g_slots[kMaxDevices];
std::mutex g_slots_mu;
// wait bound written into the status word by each call (randqr_set_wait_limit(NULL, polls))
std::atomic<int32_t> g_static_wait_field{0};

// Once per device, with that device current: the device addresses of the static arrays.
// (In host code the array names are host-side stand-ins, not device addresses.)
cudaError_t static_slot(int dev, StaticSlot *out) {
  std::lock_guard<std::mutex> lock(g_slots_mu);
  StaticSlot &s = g_slots[dev];
  if (!s.ready) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_w1);
    if (e != cudaSuccess) return e;
    s.w1 = (double *)p;
    e = cudaGetSymbolAddress(&p, g_static_status);
    if (e != cudaSuccess) return e;
    s.status = (rq::DevStatus *)p;
    e = cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    s.ready = true;
  }
  *out = s;
  return cudaSuccess;
}

}  // namespace

extern "C" randqr_status randqr_sketch_static(const double *V, int64_t m, int64_t n, int64_t ldv,
                                              int64_t s1, int64_t s2, uint64_t seed,
                                              const double *S2, double *Ws, void *stream) {
  if (!V || !S2 || !Ws || n < 1 || m < 1 || ldv < n || s2 < n || s1 < s2 ||
      s1 >= (int64_t(1) << 31) || s1 * n > kStaticW1Max)
    return RANDQR_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return RANDQR_ERR_CUDA;
  }
  StaticSlot slot;
  if (static_slot(dev, &slot) != cudaSuccess) {
    cudaGetLastError();
    return RANDQR_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // W1 and Ws accumulate with atomics and the status word gates the kernels: all three
  // must start at zero on every call (the array keeps the previous call's contents); the
  // status word also carries the wait bound.
  if (rq::launch_status_reset(slot.status, g_static_wait_field.load(), s) != cudaSuccess ||
      cudaMemsetAsync(slot.w1, 0, sizeof(double) * (size_t)(s1 * n), s) != cudaSuccess ||
      cudaMemsetAsync(Ws, 0, sizeof(double) * (size_t)(s2 * n), s) != cudaSuccess ||
      rq::launch_cs_scatter(V, m, n, ldv, s1, seed, 0, slot.w1, slot.num_sms, slot.status, s) !=
          cudaSuccess ||
      rq::launch_sketch_gemm(S2, slot.w1, s2, s1, n, Ws, true, slot.num_sms, slot.status, s) !=
          cudaSuccess) {
    cudaGetLastError();
    return RANDQR_ERR_CUDA;
  }
  return RANDQR_OK;
}

extern "C" randqr_status randqr_sketch_static_status(void *stream, randqr_info *info) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return RANDQR_ERR_CUDA;
  }
  StaticSlot slot;
  if (static_slot(dev, &slot) != cudaSuccess) {
    cudaGetLastError();
    return RANDQR_ERR_CUDA;
  }
  // a plain host variable as the destination: the copy is synchronous for pageable memory,
  // and nothing is allocated
  rq::DevStatus h;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess ||
      cudaMemcpyAsync(&h, slot.status, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return RANDQR_ERR_CUDA;
  }
  if (info) {
    info->info = h.info;
    info->stage = h.stage;
    info->rs_min_diag = h.dmin;
    info->rs_max_diag = h.dmax;
    info->orth_err2 = -1.0;
    info->resid_relF = -1.0;
  }
  return (randqr_status)h.code;
}

void rq_static_set_wait_limit(int32_t polls) {
  g_static_wait_field.store(polls < 0 ? 0 : std::min<int32_t>(polls, (1 << 30) - 1) + 1);
}
