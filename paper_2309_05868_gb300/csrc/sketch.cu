// sketch.cu -- Algorithm 1 step 1: W1 = S1 V (CountSketch), Ws = S2 W1 (Gaussian sketch).
//
// Sec. 4.2 of the paper splits the multisketch into a sparse CountSketch pass over the
// tall matrix and a small dense product.  The CountSketch never exists as a matrix here:
// each row's bucket and sign come from an integer hash computed on the fly, and the row
// is added into W1 with L2 atomics, so the pass reads V once and touches only the
// s1 x n buffer (L2-resident at every size this library accepts).
#include "common.cuh"

namespace rq {

// ---------------------------------------------------------------------------------------
// Step 1: buckets and signs, written out (used by callers who want S1 explicitly, and by
// the bit-exactness tests).
// ---------------------------------------------------------------------------------------
__global__ void k_cs_hash(uint64_t seed, int64_t m, uint32_t s1, int32_t *bucket, int8_t *sign) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t bs = cs_bucket_sign(seed, (uint64_t)i, s1);
    bucket[i] = (int32_t)(bs & 0x7fffffffu);
    sign[i] = (bs >> 31) ? (int8_t)-1 : (int8_t)1;
  }
}

cudaError_t launch_cs_hash(uint64_t seed, int64_t m, int64_t s1, int32_t *bucket, int8_t *sign,
                           cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  int blocks = (int)std::min<int64_t>(ceil_div(m, 256), 4096);
  k_cs_hash<<<blocks, 256, 0, s>>>(seed, m, (uint32_t)s1, bucket, sign);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Gaussian S2 with N(0, 1/s2) entries: Philox4x64-10 at counter (r*s1 + c) and key
// (seed, 0), Box-Muller on the first two words.
// ---------------------------------------------------------------------------------------
__global__ void k_gauss_gen(uint64_t seed, int64_t total, double scale, double *S2) {
  const double two_m53 = 1.1102230246251565404e-16;
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    uint64_t c[4] = {(uint64_t)idx, 0, 0, 0};
    philox4x64_10(c, seed, 0);
    double u1 = (double)((c[0] >> 11) + 1) * two_m53;
    double u2 = (double)(c[1] >> 11) * two_m53;
    double z = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
    S2[idx] = z * scale;
  }
}

cudaError_t launch_gauss_gen(uint64_t seed, int64_t s2, int64_t s1, double *S2, cudaStream_t s) {
  int64_t total = s2 * s1;
  int blocks = (int)std::min<int64_t>(ceil_div(total, 256), 8192);
  k_gauss_gen<<<blocks, 256, 0, s>>>(seed, total, 1.0 / sqrt((double)s2), S2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Rademacher S2 with entries +-1/sqrt(s2): entry (r, c) is negative when bit c % 64 of
// splitmix64(seed ^ splitmix64(r * ceil(s1 / 64) + c / 64)) is set.  One thread per entry.
// ---------------------------------------------------------------------------------------
__global__ void k_rad_gen(uint64_t seed, int64_t s2, int64_t s1, double scale, double *S2) {
  const int64_t total = s2 * s1, nw = (s1 + 63) / 64;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / s1, c = idx - r * s1;
    const uint64_t word = splitmix64(seed ^ splitmix64((uint64_t)(r * nw + (c >> 6))));
    S2[idx] = ((word >> (c & 63)) & 1ULL) ? -scale : scale;
  }
}

cudaError_t launch_rad_gen(uint64_t seed, int64_t s2, int64_t s1, double *S2, cudaStream_t s) {
  const int64_t total = s2 * s1;
  const int blocks = (int)std::min<int64_t>(ceil_div(total, 256), 8192);
  k_rad_gen<<<blocks, 256, 0, s>>>(seed, s2, s1, 1.0 / sqrt((double)s2), S2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// CountSketch scatter-add: W1[bucket(i), :] += sign(i) V[i, :].
// One warp takes 32 consecutive rows: each lane hashes one of them, then the warp walks the
// rows, broadcasting (bucket, sign) with a shuffle, lanes striding over the columns so the
// loads of a row are coalesced.  Rows are taken in groups of RG with all their loads issued
// before the atomics, to keep several row reads in flight per warp.  The sign is applied
// by flipping the sign bit (integer op), and the add runs as an L2 atomic (RED.ADD.F64).
// ---------------------------------------------------------------------------------------
template <int CPL>  // columns per lane: n <= 32 * CPL
__global__ void __launch_bounds__(256) k_cs_scatter(const double *__restrict__ V, int64_t m, int n,
                                                    int64_t ldv, uint32_t s1, uint64_t seed,
                                                    int64_t row0, double *__restrict__ W1,
                                                    const DevStatus *st) {
  if (status_failed(st)) return;
  constexpr int RG = 4;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = warp * 32; base < m; base += nwarps * 32) {
    const int64_t mine = base + lane;
    const uint32_t bs = (mine < m) ? cs_bucket_sign(seed, (uint64_t)(row0 + mine), s1) : 0u;
    const int rows = (int)imin64(32, m - base);
    for (int r0 = 0; r0 < rows; r0 += RG) {
      double v[RG][CPL];
#pragma unroll
      for (int g = 0; g < RG; ++g) {
        const double *vr = V + (base + r0 + g) * ldv;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int j = lane + 32 * c;
          v[g][c] = (r0 + g < rows && j < n) ? __ldg(vr + j) : 0.0;
        }
      }
#pragma unroll
      for (int g = 0; g < RG; ++g) {
        const uint32_t x = __shfl_sync(0xffffffffu, bs, (r0 + g) & 31);
        if (r0 + g < rows) {
          double *wr = W1 + (int64_t)(x & 0x7fffffffu) * n;
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const int j = lane + 32 * c;
            if (j < n) atomicAdd(wr + j, flip_if(v[g][c], x >> 31));
          }
        }
      }
    }
  }
}

// The same scatter with one bulk reduce-add per row: the warp reads the row (coalesced),
// applies the sign while writing it into a ring slot of its own in shared memory, and one lane
// hands the slot to the bulk-copy engine as an FP64 add into W1's bucket row
// (cp.reduce.async.bulk .add.f64): one request of 8 n bytes per row instead of n scalar
// reductions.  A slot is rewritten only after the engine has read it (bulk groups committed
// per row, waited for with a lag of RING - 1).  Needs 16-byte aligned rows of W1 (n even).
constexpr int SC_WARPS = 8;

__device__ __forceinline__ void bulk_reduce_add_f64(double *dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;\n" ::"l"(dst), "r"(src),
               "r"(bytes)
               : "memory");
}

template <int CPL, int RING = (CPL <= 2 ? 8 : 4)>
__global__ void __launch_bounds__(SC_WARPS * 32) k_cs_scatter_bulk(const double *__restrict__ V, int64_t m, int n,
                                                                   int64_t ldv, uint32_t s1, uint64_t seed,
                                                                   int64_t row0, double *__restrict__ W1,
                                                                   const DevStatus *st) {
  if (status_failed(st)) return;
  constexpr int RG = 4;
  __shared__ __align__(16) double ring[SC_WARPS][RING][32 * CPL];  // at most 32 KB
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t bytes = (uint32_t)n * 8u;
  int k = 0;  // rows handed to the engine by this warp
  for (int64_t base = warp * 32; base < m; base += nwarps * 32) {
    const int64_t mine = base + lane;
    const uint32_t bs = (mine < m) ? cs_bucket_sign(seed, (uint64_t)(row0 + mine), s1) : 0u;
    const int rows = (int)imin64(32, m - base);
    for (int r0 = 0; r0 < rows; r0 += RG) {
      double v[RG][CPL];
#pragma unroll
      for (int g = 0; g < RG; ++g) {
        const double *vr = V + (base + r0 + g) * ldv;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int j = lane + 32 * c;
          v[g][c] = (r0 + g < rows && j < n) ? __ldg(vr + j) : 0.0;
        }
      }
#pragma unroll
      for (int g = 0; g < RG; ++g) {
        const uint32_t x = __shfl_sync(0xffffffffu, bs, (r0 + g) & 31);
        if (r0 + g < rows) {
          double *slot = ring[wl][k % RING];
          if (k >= RING) {  // the engine has read this slot's previous row
            if (lane == 0) asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(RING - 1) : "memory");
            __syncwarp();
          }
#pragma unroll
          for (int c = 0; c < CPL; ++c) slot[lane + 32 * c] = flip_if(v[g][c], x >> 31);
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
          __syncwarp();
          if (lane == 0) {
            bulk_reduce_add_f64(W1 + (int64_t)(x & 0x7fffffffu) * n, (uint32_t)__cvta_generic_to_shared(slot), bytes);
            asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
          }
          ++k;
        }
      }
    }
  }
  if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

cudaError_t launch_cs_scatter(const double *V, int64_t m, int64_t n, int64_t ldv, int64_t s1,
                              uint64_t seed, int64_t row0, double *W1, int num_sms, const DevStatus *st,
                              cudaStream_t s) {
  if (n % 2 == 0 && n <= 128 && ((uintptr_t)W1 & 15) == 0) {
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(m, 32 * SC_WARPS), (int64_t)num_sms * 8));
    if (n <= 32)
      k_cs_scatter_bulk<1><<<blocks, SC_WARPS * 32, 0, s>>>(V, m, (int)n, ldv, (uint32_t)s1, seed, row0, W1, st);
    else if (n <= 64)
      k_cs_scatter_bulk<2><<<blocks, SC_WARPS * 32, 0, s>>>(V, m, (int)n, ldv, (uint32_t)s1, seed, row0, W1, st);
    else
      k_cs_scatter_bulk<4><<<blocks, SC_WARPS * 32, 0, s>>>(V, m, (int)n, ldv, (uint32_t)s1, seed, row0, W1, st);
    return cudaGetLastError();
  }
  int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(m, 256), (int64_t)num_sms * 8));
  if (n <= 32)
    k_cs_scatter<1><<<blocks, 256, 0, s>>>(V, m, (int)n, ldv, (uint32_t)s1, seed, row0, W1, st);
  else if (n <= 64)
    k_cs_scatter<2><<<blocks, 256, 0, s>>>(V, m, (int)n, ldv, (uint32_t)s1, seed, row0, W1, st);
  else
    k_cs_scatter<4><<<blocks, 256, 0, s>>>(V, m, (int)n, ldv, (uint32_t)s1, seed, row0, W1, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Ws = S2 W1: (s2 x s1)(s1 x n).  FP64 tiles of 64 x 64 outputs, 4 x 4 per thread, K
// staged through shared memory in slices of 16, and the long K = s1 split across CTAs
// (split-K) so the whole GPU works on it; partial tiles are summed with L2 atomics into
// a zeroed Ws.
// ---------------------------------------------------------------------------------------
constexpr int GB = 64, GK = 16;
__global__ void __launch_bounds__(256) k_sketch_gemm(const double *__restrict__ S2,
                                                     const double *__restrict__ W1, int s2,
                                                     int64_t s1, int n, double *__restrict__ Ws,
                                                     int64_t kchunk, const DevStatus *st) {
  if (status_failed(st)) return;
  __shared__ double As[GK][GB + 1];
  __shared__ double Bs[GK][GB + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = blockIdx.y * GB, c0 = blockIdx.x * GB;
  const int64_t kb = blockIdx.z * kchunk;
  const int64_t ke = imin64(s1, kb + kchunk);
  double acc[4][4] = {};
  for (int64_t k0 = kb; k0 < ke; k0 += GK) {
    for (int e = threadIdx.x; e < GB * GK; e += 256) {
      const int rr = e / GK, kk = e % GK;
      const int64_t gr = r0 + rr, gk = k0 + kk;
      As[kk][rr] = (gr < s2 && gk < ke) ? S2[gr * s1 + gk] : 0.0;
      const int kk2 = e / GB, cc = e % GB;
      const int64_t gk2 = k0 + kk2, gc = c0 + cc;
      Bs[kk2][cc] = (gk2 < ke && gc < n) ? W1[gk2 * n + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gr = r0 + ty * 4 + i, gc = c0 + tx * 4 + j;
      if (gr < s2 && gc < n) atomicAdd(Ws + (int64_t)gr * n + gc, acc[i][j]);
    }
}

cudaError_t launch_sketch_gemm(const double *S2, const double *W1, int64_t s2, int64_t s1,
                               int64_t n, double *Ws, bool use_tc, int num_sms, DevStatus *st,
                               cudaStream_t s) {
  if (use_tc && sketch_oz_supported(n)) return launch_sketch_oz(S2, s1, W1, n, s2, s1, n, Ws, num_sms, st, s);
  const int64_t tiles = ceil_div(s2, GB) * ceil_div(n, GB);
  int64_t split = std::max<int64_t>(1, (2 * (int64_t)num_sms) / tiles);
  split = std::min<int64_t>(split, ceil_div(s1, GK));
  int64_t kchunk = ceil_div(ceil_div(s1, split), GK) * GK;
  split = ceil_div(s1, kchunk);
  dim3 grid((unsigned)ceil_div(n, GB), (unsigned)ceil_div(s2, GB), (unsigned)split);
  k_sketch_gemm<<<grid, 256, 0, s>>>(S2, W1, (int)s2, s1, (int)n, Ws, kchunk, st);
  return cudaGetLastError();
}

}  // namespace rq
